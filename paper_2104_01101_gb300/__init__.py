"""GB300-native sketched Tucker-ALS (Ma & Solomonik, arXiv 2104.01101).

The compute path is the CUDA library ``libtsketch.so`` (sources in ``csrc/``,
C-ABI declared in ``include/tsketch.h``).  ``paper_2104_01101_gb300.tsketch`` is
its thin Python binding (argument marshalling only); importing it fails loudly
when the library has not been built.  ``synth`` generates seeded inputs.
"""

__all__ = ["synth", "tsketch"]
