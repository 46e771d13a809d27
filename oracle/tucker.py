"""Drivers of the sketched Tucker method and its reference algorithms, FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Contents: fitness (Sec. 7), HOSVD and HOOI (Sec. 2.2, Alg. 1), Init-RRF with the
composite sketch (Alg. 3, Sec. 5), Sketch-Tucker-ALS (Alg. 4) with TensorSketch
or leverage-score sampling and either solve of ``oracle.solve``, CP-ALS (Alg. 2)
and CP-Sketch-Tucker (Alg. 6).
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import rng
from .sketch import (input_sketch_coo, input_sketch_dense, leverage_sketch_coo,
                     leverage_sketch_coo_det, leverage_sketch_dense, leverage_sketch_dense_det,
                     ts_apply_fft, ts_tables_for_mode)
from .solve import canonical_signs, lrls_exact, rsvd_lrls, rsvd_oversampled_rank
from .tensor import fold, kron_chain, reconstruct, ttm, unfold


@dataclass
class Coo:
    """Sparse tensor: idx is (N, nnz) integer coordinates, vals the values; duplicates add."""
    idx: np.ndarray
    vals: np.ndarray
    dims: tuple

    @property
    def ndim(self):
        return len(self.dims)


def dims_of(X):
    return tuple(X.dims) if isinstance(X, Coo) else tuple(X.shape)


# --------------------------------------------------------------------------
# Fitness (Sec. 7)
# --------------------------------------------------------------------------

def coo_norm2(X: Coo) -> float:
    """||T||_F^2 of a COO tensor, summing duplicate coordinates first."""
    order = np.lexsort(X.idx[::-1])
    idx = X.idx[:, order]
    v = X.vals[order].astype(np.float64)
    new = np.ones(v.shape[0], dtype=bool)
    new[1:] = np.any(idx[:, 1:] != idx[:, :-1], axis=0)
    sums = np.add.reduceat(v, np.flatnonzero(new))
    return float(np.dot(sums, sums))


def coo_inner_with_tucker(X: Coo, core, factors) -> float:
    """<T, C x_1 A^(1) ... x_N A^(N)> = sum over stored entries of v * T~(i)."""
    total = 0.0
    chunk = 1 << 15
    for a in range(0, X.vals.shape[0], chunk):
        b = min(a + chunk, X.vals.shape[0])
        N = X.ndim
        rows = [factors[n][X.idx[n, a:b]] for n in range(N)]       # (chunk, R_n)
        G = np.einsum("...r,cr->c...", core, rows[N - 1])          # contract mode N
        for n in range(N - 2, -1, -1):                             # then N-1, ..., 1
            G = np.einsum("c...r,cr->c...", G, rows[n])
        total += float(np.dot(G, X.vals[a:b].astype(np.float64)))
    return total


def tucker_norm2(core, factors) -> float:
    """||C x_1 A^(1) ... ||^2 = <C, C x_1 (A^(1)T A^(1)) ...> (exact without orthonormality)."""
    G = core
    for n, A in enumerate(factors):
        G = ttm(G, A.T @ A, n)
    return float(np.sum(G * core))


def residual(X, core, factors) -> float:
    """||T - T~||_F / ||T||_F, i.e. 1 - fitness."""
    if isinstance(X, Coo):
        t2 = coo_norm2(X)
        r2 = t2 - 2.0 * coo_inner_with_tucker(X, core, factors) + tucker_norm2(core, factors)
        return math.sqrt(max(r2, 0.0) / t2)
    Xt = reconstruct(core, factors)
    return float(np.linalg.norm(X - Xt) / np.linalg.norm(X))


def fitness(X, core, factors) -> float:
    """f = 1 - ||T - T~||_F / ||T||_F (Sec. 7)."""
    return 1.0 - residual(X, core, factors)


# --------------------------------------------------------------------------
# HOSVD and HOOI (Sec. 2.2, Alg. 1)
# --------------------------------------------------------------------------

def leading_left_singular_vectors(M: np.ndarray, R: int) -> np.ndarray:
    U, _, _ = np.linalg.svd(M, full_matrices=False)
    U = U[:, :R]
    _, U = canonical_signs(np.zeros((1, R)), U)
    return U


def hosvd(T: np.ndarray, ranks):
    """A^(n) = leading R_n left singular vectors of T_(n) (Sec. 2.2)."""
    return [leading_left_singular_vectors(unfold(T, n), R) for n, R in enumerate(ranks)]


def hooi(T: np.ndarray, ranks, sweeps: int, init=None):
    """Tucker-ALS / HOOI, Alg. 1, with HOSVD initialisation unless ``init`` is given."""
    N = T.ndim
    A = [a.copy() for a in init] if init is not None else hosvd(T, ranks)
    core = None
    for _ in range(sweeps):
        for n in range(N):
            Yt = T
            for k in range(N):
                if k != n:
                    Yt = ttm(Yt, A[k].T, k)
            A[n] = leading_left_singular_vectors(unfold(Yt, n), ranks[n])
        core = ttm(Yt, A[N - 1].T, N - 1)
    return core, A


# --------------------------------------------------------------------------
# Init-RRF (Alg. 3) with the composite sketch (Sec. 5)
# --------------------------------------------------------------------------

def rrf_sizes(dims, n: int, R: int, m: int, k1=None, k2=None):
    """(k1, k2) of the composite sketch for mode n.

    Reading: k1 = ceil(sqrt(K) R) with K = m / R^2 (Sec. 7 sets the RRF sketch size
    to sqrt(K) R), unless given; k2 = R^2 + k1 (the definition's O(R^2 + R/eps));
    both clipped to the sizes of T_(n).
    """
    K = int(np.prod([dims[k] for k in range(len(dims)) if k != n]))
    if k1 is None or k1 <= 0:
        k1 = int(math.ceil(math.sqrt(m)))
    if k2 is None or k2 <= 0:
        k2 = R * R + k1
    k2 = min(k2, K)
    k1 = max(R, min(k1, k2, dims[n]))
    return k1, k2


def rrf_tables(seed: int, dims, n: int, k2: int):
    return [rng.hash_table(seed, rng.PURPOSE_RRF_HASH, 0, n, k, dims[k], k2)
            for k in range(len(dims)) if k != n]


def rrf_gaussian(seed: int, n: int, k1: int, k2: int) -> np.ndarray:
    """G in R^{k2 x k1} with N(0, 1/k1) entries (composite sketching matrix definition)."""
    g = rng.gaussian(seed, rng.make_tag(rng.PURPOSE_RRF_GAUSS, 0, n, 0), k2 * k1)
    return g.reshape(k2, k1) / math.sqrt(k1)


def init_rrf(X, n: int, R: int, k1: int, k2: int, seed: int) -> np.ndarray:
    """Alg. 3 on M = T_(n): B = M S with S = T G composite, U = svd(B), return U(:, :R).

    Reading: the CountSketch factor T (over the prod_{k != n} s_k columns of T_(n),
    k2 buckets) uses the restricted TensorSketch hash of Sec. 3.1 with its own
    tables, which satisfies the CountSketch definition's Pr[h(i) = j] = 1/k2, so
    B = (S' T_(n)^T)^T G.
    """
    dims = dims_of(X)
    tables = rrf_tables(seed, dims, n, k2)
    if isinstance(X, Coo):
        Wt = input_sketch_coo(X.idx, X.vals, dims, n, tables, k2)
    else:
        Wt = input_sketch_dense(X, n, tables, k2)
    B = Wt.T @ rrf_gaussian(seed, n, k1, k2)
    return leading_left_singular_vectors(B, R)


# --------------------------------------------------------------------------
# Sketch-Tucker-ALS (Alg. 4)
# --------------------------------------------------------------------------

def sketch_tucker_als(X, ranks, m: int, sweeps: int, seed: int, kind: str = "ts",
                      solve: str = "rsvd", oversample: int = 5, rrf_k1=None, rrf_k2=None,
                      resketch: bool = False, init_factors=None, ts_tables=None,
                      track_fit: bool = False):
    """Alg. 4.  Returns (core, factors, per-sweep residuals or []).

    kind       "ts" (TensorSketch, RHS sketch built once and reused across sweeps
               unless ``resketch``), "lev" (leverage-score sampling, redrawn for every
               subproblem) or "lev_det" (the m rows of largest leverage score,
               reselected for every subproblem); the leverage kinds gather the sampled
               fibres of a COO tensor from its nonzeros.
    solve      "rsvd" (Alg. 5, the routine Alg. 4 calls) or "exact" (the solution
               Theorem 4.1 is stated for).
    init_factors  replaces the RRF initialisation of modes 2..N when given.
    ts_tables  optional {n: [(bins, signs) for k != n]} replacing the hashed tables.
    """
    dims = dims_of(X)
    N = len(dims)
    assert N >= 2 and len(ranks) == N
    factors = [None] * N
    if init_factors is not None:
        factors = [None if a is None else np.array(a, dtype=np.float64) for a in init_factors]
    else:
        for n in range(1, N):
            k1, k2 = rrf_sizes(dims, n, ranks[n], m, rrf_k1, rrf_k2)
            factors[n] = init_rrf(X, n, ranks[n], k1, k2, seed)
    core = np.zeros(ranks)
    y_cache = {}
    fits = []
    for sweep in range(sweeps):
        for n in range(N):
            others = [k for k in range(N) if k != n]
            if kind == "ts":
                tsweep = sweep if resketch else 0
                tables = ts_tables[n] if ts_tables is not None else \
                    ts_tables_for_mode(seed, dims, n, m, tsweep)
                key = (n, tsweep)
                if key not in y_cache:
                    if isinstance(X, Coo):
                        y_cache[key] = input_sketch_coo(X.idx, X.vals, dims, n, tables, m)
                    else:
                        y_cache[key] = input_sketch_dense(X, n, tables, m)
                Y = y_cache[key]
                Z = ts_apply_fft([factors[k] for k in others], tables, m)
            elif kind == "lev":
                if isinstance(X, Coo):
                    Z, Y, _, _ = leverage_sketch_coo(X.idx, X.vals, dims, n, factors, m, seed,
                                                     sweep)
                else:
                    Z, Y, _, _ = leverage_sketch_dense(X, n, factors, m, seed, sweep)
            elif kind == "lev_det":
                if isinstance(X, Coo):
                    Z, Y, _ = leverage_sketch_coo_det(X.idx, X.vals, dims, n, factors, m)
                else:
                    Z, Y, _ = leverage_sketch_dense_det(X, n, factors, m)
            else:
                raise ValueError(kind)
            if solve == "exact":
                CnT, An = lrls_exact(Z, Y, ranks[n])
            else:
                r = Z.shape[1]
                k = rsvd_oversampled_rank(ranks[n], oversample, r, dims[n])
                Omega = rng.gaussian(seed, rng.make_tag(rng.PURPOSE_RSVD_GAUSS, sweep, n, 0),
                                     dims[n] * k).reshape(dims[n], k)
                CnT, An = rsvd_lrls(Z, Y, ranks[n], Omega)
            factors[n] = An
            core = fold(CnT.T, n, ranks)
        if track_fit:
            fits.append(residual(X, core, factors))
    return core, factors, fits


# --------------------------------------------------------------------------
# CP-ALS (Alg. 2) and CP-Sketch-Tucker (Alg. 6)
# --------------------------------------------------------------------------

def khatri_rao(mats) -> np.ndarray:
    """Column-wise Kronecker product, first factor slowest (Sec. 2.1)."""
    out = np.ones((1, mats[0].shape[1]))
    for A in mats:
        out = (out[:, None, :] * A[None, :, :]).reshape(-1, A.shape[1])
    return out


def cp_reconstruct(factors) -> np.ndarray:
    R = factors[0].shape[1]
    T = 0.0
    for r in range(R):
        t = factors[0][:, r]
        for A in factors[1:]:
            t = np.multiply.outer(t, A[:, r])
        T = T + t
    return T


def cp_als(X: np.ndarray, R: int, sweeps: int, init):
    """Alg. 2: each A^(n) solves eq. (subproblem) by the normal equations (MTTKRP)."""
    N = X.ndim
    A = [a.copy() for a in init]
    for _ in range(sweeps):
        for n in range(N):
            others = [k for k in range(N) if k != n]
            P = khatri_rao([A[k] for k in others])
            gram = np.ones((R, R))
            for k in others:
                gram = gram * (A[k].T @ A[k])
            A[n] = (unfold(X, n) @ P) @ np.linalg.pinv(gram)
    return A


def cp_init_hosvd(core: np.ndarray, R: int):
    """CP initialisation by HOSVD of the core (Sec. 7.2): leading R left singular vectors."""
    return [leading_left_singular_vectors(unfold(core, n), R) for n in range(core.ndim)]


def cp_sketch_tucker(X, R: int, tucker_ranks, m: int, tucker_sweeps: int, cp_sweeps: int,
                     seed: int, **tucker_kw):
    """Alg. 6: sketched Tucker-ALS, CP-ALS on the core, factors B^(n) A^(n)."""
    core, B, _ = sketch_tucker_als(X, tucker_ranks, m, tucker_sweeps, seed, **tucker_kw)
    A = cp_als(core, R, cp_sweeps, cp_init_hosvd(core, R))
    return [B[n] @ A[n] for n in range(len(B))], core, B, A


def kron_P(factors, n):
    """P^(n) of eq. (tucker_ls), formed explicitly (small sizes only)."""
    return kron_chain([factors[k] for k in range(len(factors)) if k != n])
