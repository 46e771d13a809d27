"""Element-wise error bounds used by the GPU parity tests (computed with the oracle).

Every bound is "c * u * (a magnitude)" where the magnitude is the same computation run
on absolute values with unit signs (the sum of |terms| of each output entry), or, for
the FFT path, a per-column quantity that bounds every entry of the column.
"""

from __future__ import annotations

import numpy as np

from oracle import sketch

U32 = 2.0 ** -24  # unit roundoff of FP32 (round to nearest)
U64 = 2.0 ** -53


def unit_tables(tables):
    return [(b, np.ones_like(s)) for b, s in tables]


def input_sketch_terms(T, n, tables, m):
    """(sum of |terms|, number of terms) of every entry of Y = S T_(n)^T (dense T)."""
    absY = sketch.input_sketch_dense(np.abs(T).astype(np.float64), n, unit_tables(tables), m)
    cnt = sketch.input_sketch_dense(np.ones(T.shape), n, unit_tables(tables), m)
    return absY, cnt


def input_sketch_coo_terms(idx, vals, dims, n, tables, m):
    """The same for a COO tensor (repeated coordinates are separate terms)."""
    absY = sketch.input_sketch_coo(idx, np.abs(vals).astype(np.float64), dims, n,
                                   unit_tables(tables), m)
    cnt = sketch.input_sketch_coo(idx, np.ones(vals.shape[0]), dims, n, unit_tables(tables), m)
    return absY, cnt


def summation_bound(absY, cnt, u):
    """Any-order summation of n terms: |computed - exact| <= n u sum|terms| (first order);
    twice that between two computations that each round (the GPU's and the oracle's)."""
    return 2 * cnt * u * absY


def ts_fft_column_bound(factors, tables, m, u):
    """Per-column bound on every entry of Z = IFFT(prod FFT(U_f)) with U_f = S_f A_f.

    A circular convolution by FFTs of length m has normwise error at most about
    c u log2(m) prod_f ||U_f[:, c_f]||_1 (each transform is a product of log2(m)
    butterfly stages, each a rounding error relative to the 1-norm of its input), and
    max_i |err_i| <= ||err||_2; the direct CountSketch adds n_f roundings per entry.  c = 4
    covers the complex products; the bound is the same for every entry of a column.
    """
    norms = []
    for A, (bins, signs) in zip(factors, tables):
        U = sketch.countsketch_matrix(bins, np.ones_like(signs), m) @ np.abs(A)
        norms.append(U.sum(axis=0))  # ||U_f[:, r]||_1 with unit signs: an upper bound
    col = np.ones(1)
    for nv in norms:
        col = (col[:, None] * nv[None, :]).reshape(-1)
    c = 4.0 * (np.log2(m) + len(factors) + 2)
    return c * u * col[None, :]


def fit_grad_abs(core, factors, Y, tables, n, m):
    """The sketched-fit gradient chain of oracle.grad run on absolute values (|S|, |P|,
    |C|, |A|) with the residual's terms added in magnitude (|Z||M| + |Y|): every entry
    bounds the sum of |terms| that forms the matching entry of the gradient."""
    from oracle.tensor import fold, kron_chain, unfold
    N = len(factors)
    others = [k for k in range(N) if k != n]
    S = sketch.tensorsketch_dense(unit_tables(tables), m)
    Ab = [np.abs(f) for f in factors]
    P = kron_chain([Ab[k] for k in others])
    Z = S @ P
    Cn = np.abs(unfold(core, n))
    M = Cn.T @ Ab[n].T
    R = Z @ M + np.abs(Y)
    gA = [None] * N
    gA[n] = R.T @ Z @ Cn.T
    gcore = fold((Z.T @ R @ Ab[n]).T, n, core.shape)
    dP = S.T @ R @ M.T
    rows = [factors[k].shape[0] for k in others]
    cols = [factors[k].shape[1] for k in others]
    q = len(others)
    D = dP.reshape(rows + cols)
    low, up = "abcdefgh"[:q], "ABCDEFGH"[:q]
    for a, k in enumerate(others):
        terms = [low + up] + [low[b] + up[b] for b in range(q) if b != a]
        ops = [D] + [Ab[others[b]] for b in range(q) if b != a]
        gA[k] = np.einsum(",".join(terms) + "->" + low[a] + up[a], *ops)
    return gcore, gA


def fit_grad_depth(dims, ranks, n, m):
    """Roundings along the longest chain of the gradient (first order): the FFT of each
    factor chain (4 log2 m), the residual (r = prod_{k != n} R_k products, then one
    subtraction), the products with Z^T (m terms) and with the core or the other
    factors (r or s_n terms), the adjoint FFT (4 log2 m)."""
    r = int(np.prod([R for k, R in enumerate(ranks) if k != n]))
    return 8 * np.log2(m) + 2 * r + m + max(dims) + ranks[n] + 8
