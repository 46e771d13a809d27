"""FP64 CPU oracle for the sketched Tucker-ALS hot path (Ma & Solomonik, arXiv 2104.01101).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, deliberately obvious
restatement of what the paper computes, written in numpy/scipy FP64.  It exists
to check the CUDA library; it is never part of the product path.  Only the test
suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  It shares no code with the CUDA path and
imports nothing from the ``paper_2104_01101_gb300`` package.

Modules
-------
rng      counter-based random numbers (splitmix64) and the polynomial hash family
         that realises the paper's 3-/4-wise independent hash maps (Sec. 3.1).
sketch   CountSketch / TensorSketch definitions, the FFT identity for SP,
         the one-pass sketch of the data tensor, leverage-score sampling on dense and
         COO tensors, random and deterministic (Sec. 3).
solve    the sketched rank-constrained least-squares solves: the exact form of
         Theorem 4.1's definition and RSVD-LRLS (Alg. 5).
tucker   unfolding/TTM helpers, fitness (Sec. 7), HOSVD + HOOI (Alg. 1),
         Init-RRF (Alg. 3), Sketch-Tucker-ALS (Alg. 4), CP-ALS (Alg. 2) and
         CP-Sketch-Tucker (Alg. 6).
grad     the sketched fit of one subproblem and its gradient with respect to the
         core and every factor, by explicit matrices and the chain rule.

Parity status: every function here is pinned by a ``-m "not gpu"`` test against
something other than itself (brute force, closed forms, invariants, HOOI
equivalence); none is "parity unpinned".
"""

from . import grad, rng, sketch, solve, tucker  # noqa: F401
