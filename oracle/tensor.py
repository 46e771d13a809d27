"""Tensor-algebra helpers in the paper's notation (Sec. 2.1), FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Index-order convention (a reading of the paper, which linearises multi-indices
with the first index fastest in Sec. 3.1 but writes Kronecker chains in the
standard first-factor-slowest order in Sec. 2.2): C order everywhere.

* mode-n unfolding  T_(n) = moveaxis(T, n, 0).reshape(s_n, -1); its columns run
  over the remaining modes in ascending order, last mode fastest;
* P^(n) = A^(1) (x) ... (x) A^(n-1) (x) A^(n+1) (x) ... (x) A^(N) with numpy's
  ``kron`` (first factor slowest), so that T_(n)^T ~= P^(n) C_(n)^T A^(n)T.
"""

from __future__ import annotations

import numpy as np


def unfold(T: np.ndarray, n: int) -> np.ndarray:
    """Mode-n matricisation T_(n) in R^{s_n x prod_{k != n} s_k}."""
    return np.moveaxis(T, n, 0).reshape(T.shape[n], -1)


def fold(M: np.ndarray, n: int, shape) -> np.ndarray:
    """Inverse of :func:`unfold`."""
    rest = [shape[k] for k in range(len(shape)) if k != n]
    return np.moveaxis(M.reshape([shape[n]] + rest), 0, n)


def ttm(T: np.ndarray, M: np.ndarray, n: int) -> np.ndarray:
    """Mode-n tensor-times-matrix T x_n M with M in R^{J x s_n} (Sec. 2.1)."""
    shape = list(T.shape)
    out = M @ unfold(T, n)
    shape[n] = M.shape[0]
    return fold(out, n, shape)


def kron_chain(mats) -> np.ndarray:
    """A^(1) (x) A^(2) (x) ... with the first factor's index slowest."""
    out = np.ones((1, 1))
    for A in mats:
        out = np.kron(out, A)
    return out


def reconstruct(core: np.ndarray, factors) -> np.ndarray:
    """C x_1 A^(1) x_2 ... x_N A^(N)."""
    T = core
    for n, A in enumerate(factors):
        T = ttm(T, A, n)
    return T
