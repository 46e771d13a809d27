"""Gradient of the sketched fit of one subproblem, FP64, by explicit matrices.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Each step of Sketch-Tucker-ALS (Alg. 4) minimises, over A^(n) and the core, the
sketched least-squares objective of eq. (tucker_ls) with the TensorSketch S^(n) of
Sec. 3.1 applied on the left:

    L_n(C, A^(1..N)) = 1/2 || S^(n) P^(n) C_(n)^T A^(n)T - Y ||_F^2 ,
    P^(n) = kron_{k != n} A^(k),   Y = S^(n) T_(n)^T  (the sketched right-hand side).

Its gradient with respect to the core and to every factor (the factors k != n enter
through P^(n)) is written out below with S^(n) and P^(n) formed explicitly, by the
chain rule on the matrix products: no FFT, no structure, small sizes only.
"""

from __future__ import annotations

import numpy as np

from .sketch import tensorsketch_dense
from .tensor import fold, kron_chain, unfold


def sketched_fit(core, factors, Y, tables, n: int, m: int) -> float:
    """L_n: ``tables`` are the (bins, signs) of the modes k != n, ascending."""
    N = len(factors)
    S = tensorsketch_dense(tables, m)
    P = kron_chain([factors[k] for k in range(N) if k != n])
    R = S @ P @ unfold(core, n).T @ factors[n].T - Y
    return 0.5 * float(np.sum(R * R))


def sketched_fit_grad(core, factors, Y, tables, n: int, m: int):
    """(L_n, dL/dcore, [dL/dA^(k) for every k]).

    With Z = S P, M = C_(n)^T A^(n)T and R = Z M - Y:
      dL/dA^(n)   = R^T Z C_(n)^T
      dL/dC_(n)   = (Z^T R A^(n))^T                     (folded back to the core)
      dL/dP       = S^T R M^T,  and for P = kron of the k != n factors,
      dL/dA^(k)[i_k, r_k] = sum over the other indices of dL/dP[(i), (r)] times the
                            product of the other factors' entries A^(j)[i_j, r_j].
    """
    N = len(factors)
    others = [k for k in range(N) if k != n]
    S = tensorsketch_dense(tables, m)
    P = kron_chain([factors[k] for k in others])
    Z = S @ P
    Cn = unfold(core, n)
    M = Cn.T @ factors[n].T
    R = Z @ M - Y
    loss = 0.5 * float(np.sum(R * R))
    gA = [None] * N
    gA[n] = R.T @ Z @ Cn.T
    gcore = fold((Z.T @ R @ factors[n]).T, n, core.shape)
    dP = S.T @ R @ M.T
    # dP indexed as (i_1 .. i_q, r_1 .. r_q) over the k != n factors, C order
    rows = [factors[k].shape[0] for k in others]
    cols = [factors[k].shape[1] for k in others]
    q = len(others)
    D = dP.reshape(rows + cols)
    low, up = "abcdefgh"[:q], "ABCDEFGH"[:q]
    for a, k in enumerate(others):
        terms = [low + up] + [low[b] + up[b] for b in range(q) if b != a]
        ops = [D] + [factors[others[b]] for b in range(q) if b != a]
        gA[k] = np.einsum(",".join(terms) + "->" + low[a] + up[a], *ops)
    return loss, gcore, gA
