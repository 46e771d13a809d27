"""Sketching operators of Sec. 3 (TensorSketch, leverage-score sampling), FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Conventions (readings of the paper):

* 0-based buckets: the paper's (sum_n (H_n(i_n) - 1) mod m) + 1 (Sec. 3.1,
  TensorSketch definition) is written here as (sum_n H_n(i_n)) mod m.
* A "table set" for a TensorSketch over modes k_1 < k_2 < ... is a list of
  (bins, signs) pairs, one per sketched mode, in ascending mode order.
* Row multi-indices of a Kronecker chain / unfolding are in C order (see
  ``oracle.tensor``).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import rng
from .tensor import kron_chain, unfold


# --------------------------------------------------------------------------
# CountSketch and TensorSketch (Sec. 3.1)
# --------------------------------------------------------------------------

def countsketch_matrix(bins: np.ndarray, signs: np.ndarray, m: int) -> np.ndarray:
    """Dense S = Omega D in R^{m x n} of the CountSketch definition (Sec. 3.1).

    Omega(j, i) = 1 iff j = h(i); D = diag(signs).
    """
    n = bins.shape[0]
    Omega = np.zeros((m, n))
    Omega[bins, np.arange(n)] = 1.0
    return Omega * np.asarray(signs, dtype=np.float64)[None, :]  # Omega D, D diagonal


def ts_hash(tables, m: int):
    """Bucket H(i) and sign S(i) of every multi-index (C order) of a TensorSketch.

    H(i_1..i_q) = (sum_j H_j(i_j)) mod m,  S(i_1..i_q) = prod_j S_j(i_j)
    (Sec. 3.1, the two restricted hash maps).
    """
    H = np.zeros(1, dtype=np.int64)
    S = np.ones(1)
    for bins, signs in tables:
        H = (H[:, None] + bins[None, :]).reshape(-1)
        S = (S[:, None] * signs[None, :]).reshape(-1)
    return H % m, S


def tensorsketch_sparse(tables, m: int) -> sp.csr_matrix:
    """The TensorSketch matrix S = Omega D (m x prod s_j) as an explicit sparse matrix."""
    H, S = ts_hash(tables, m)
    ncol = H.shape[0]
    return sp.csr_matrix((S, (H, np.arange(ncol))), shape=(m, ncol))


def tensorsketch_dense(tables, m: int) -> np.ndarray:
    return tensorsketch_sparse(tables, m).toarray()


def ts_apply_explicit(factors, tables, m: int) -> np.ndarray:
    """SP with P = kron of the factors formed explicitly (brute force, small sizes)."""
    P = kron_chain(factors)
    return tensorsketch_sparse(tables, m) @ P


def ts_apply_fft(factors, tables, m: int) -> np.ndarray:
    """SP by the FFT identity of Sec. 3.1.

    SP = IFFT( ( (.)_n FFT(S^(n) A^(n))^T )^T ): each factor is CountSketched to
    U_n = S^(n) A^(n) (m x R_n), transformed along its m rows, the spectra are
    combined by the row-wise Kronecker (face-splitting) product over the column
    multi-index (first factor slowest), and the result is inverse transformed.
    """
    spectra = []
    for A, (bins, signs) in zip(factors, tables):
        U = countsketch_matrix(bins, signs, m) @ A
        spectra.append(np.fft.fft(U, axis=0))
    prod = np.ones((m, 1), dtype=np.complex128)
    for F in spectra:
        prod = (prod[:, :, None] * F[:, None, :]).reshape(m, -1)
    return np.real(np.fft.ifft(prod, axis=0))


def input_sketch_dense(T: np.ndarray, n: int, tables, m: int) -> np.ndarray:
    """Y = S^(n) T_(n)^T in R^{m x s_n} (Alg. 4, sketch of the right-hand side).

    ``tables`` covers every mode k != n in ascending order.  Alg. 4 prints
    S^(n) T_(n); the dimensions of the subproblem (tucker_ls) require the
    transpose, which is what is computed.
    """
    S = tensorsketch_sparse(tables, m)
    return np.asarray(S @ unfold(T, n).T)


def input_sketch_coo(idx: np.ndarray, vals: np.ndarray, dims, n: int, tables, m: int) -> np.ndarray:
    """Y = S^(n) T_(n)^T for a COO tensor (duplicates add, the sketch is linear).

    For every nonzero (i, v): Y[(sum_{k != n} H_k(i_k)) mod m, i_n] += prod S_k(i_k) * v.
    """
    N = len(dims)
    others = [k for k in range(N) if k != n]
    b = np.zeros(vals.shape[0], dtype=np.int64)
    s = np.ones(vals.shape[0])
    for k, (bins, signs) in zip(others, tables):
        b += bins[idx[k]]
        s *= signs[idx[k]]
    Y = np.zeros((m, dims[n]))
    np.add.at(Y, (b % m, idx[n].astype(np.int64)), s * vals.astype(np.float64))
    return Y


def ts_tables_for_mode(seed: int, dims, n: int, m: int, sweep: int = 0):
    """The tables H_{n,k}, S_{n,k} (k != n, ascending) of subproblem n."""
    return [rng.hash_table(seed, rng.PURPOSE_TS_HASH, sweep, n, k, dims[k], m)
            for k in range(len(dims)) if k != n]


# --------------------------------------------------------------------------
# Leverage-score sampling (Sec. 3.2)
# --------------------------------------------------------------------------

def leverage_scores(A: np.ndarray) -> np.ndarray:
    """l_i(A) = ||Q(i,:)||_2^2 (leverage-score definition, Sec. 3.2).

    In Tucker-ALS every factor has orthonormal columns, so Q = A is an orthogonal
    basis of its column space.  The squares are added in ascending column order.
    """
    ell = np.zeros(A.shape[0])
    for r in range(A.shape[1]):
        ell = ell + A[:, r] * A[:, r]
    return ell


def leverage_sample_mode(ell: np.ndarray, u: np.ndarray):
    """Draw one index per uniform with probability ell_i / sum(ell).

    Inverse CDF: the smallest i with cdf_i > u * cdf_last, with cdf the running
    sum of ell in index order.  Returns (indices, probabilities of the drawn rows).
    """
    cdf = np.cumsum(ell)
    total = cdf[-1]
    idx = np.searchsorted(cdf, u * total, side="right")
    idx = np.minimum(idx, ell.shape[0] - 1)
    return idx, ell[idx] / total


def leverage_select_det(scores_per_mode, m: int) -> np.ndarray:
    """Deterministic leverage selection (the "Lev-fix" variant of Sec. 3.2): the m
    multi-indices with the largest Kronecker score prod_k l_k(i_k), ties broken by the
    lower C-order linear index; returned in ascending linear index."""
    sc = np.ones(1)
    for ell in scores_per_mode:
        sc = (sc[:, None] * ell[None, :]).reshape(-1)
    m = min(m, sc.shape[0])
    order = np.lexsort((np.arange(sc.shape[0]), -sc))  # score descending, index ascending
    return np.sort(order[:m])


def leverage_sketch_dense_det(T: np.ndarray, n: int, factors, m: int):
    """Sketched LHS and RHS of subproblem n by deterministic leverage sampling: the rows
    of P^(n) and the fibres of T at the multi-indices of leverage_select_det, without
    rescaling.  Returns Z (m x prod R_k), Y (m x s_n) and the multi-indices."""
    N = T.ndim
    others = [k for k in range(N) if k != n]
    lin = leverage_select_det([leverage_scores(factors[k]) for k in others], m)
    samples = np.stack(np.unravel_index(lin, [T.shape[k] for k in others]), axis=1)
    Z = kron_rows(factors, others, samples)
    Tn = np.moveaxis(T, n, -1)
    Y = Tn[tuple(samples[:, j] for j in range(len(others)))]
    return Z, Y, samples


def leverage_draws(dims, n: int, factors, m: int, seed: int, sweep: int):
    """The m leverage-score draws of subproblem n (Sec. 3.2).

    Lemma (Kronecker leverage scores, Sec. 3.2): the score of row (i_k)_{k != n} of
    P^(n) is prod_k l_{i_k}(A^(k)), so each i_k is drawn independently with
    p^(k) = l(A^(k)) / R_k, m times with replacement.  Returns the multi-indices
    (m x (N-1)) and the weights 1 / sqrt(m p_j), p_j = prod_k p^(k)_{i_k}
    (importance-sampling definition).
    """
    others = [k for k in range(len(dims)) if k != n]
    samples = np.zeros((m, len(others)), dtype=np.int64)
    prob = np.ones(m)
    for j, k in enumerate(others):
        u = rng.uniform01(seed, rng.make_tag(rng.PURPOSE_LEV_UNIFORM, sweep, n, k),
                          np.arange(m, dtype=np.uint64))
        i_k, p_k = leverage_sample_mode(leverage_scores(factors[k]), u)
        samples[:, j] = i_k
        prob = prob * p_k
    return samples, 1.0 / np.sqrt(m * prob)


def kron_rows(factors, others, samples: np.ndarray) -> np.ndarray:
    """Rows ``samples`` of P^(n) = kron of the factors of modes ``others``: entry (j, c)
    is the product of A^(k)(i_k, c_k) over the modes, first mode slowest in c."""
    Z = np.ones((samples.shape[0], 1))
    for j, k in enumerate(others):
        rows = factors[k][samples[:, j], :]
        Z = (Z[:, :, None] * rows[:, None, :]).reshape(samples.shape[0], -1)
    return Z


def leverage_sketch_dense(T: np.ndarray, n: int, factors, m: int, seed: int, sweep: int):
    """Sketched LHS and RHS of subproblem n by leverage-score sampling (leverage_draws).
    Row j of both is rescaled by its weight.  Returns Z (m x prod R_k), Y (m x s_n),
    the sampled multi-indices (m x (N-1)) and the weights.
    """
    N = T.ndim
    others = [k for k in range(N) if k != n]
    samples, w = leverage_draws(T.shape, n, factors, m, seed, sweep)
    Z = kron_rows(factors, others, samples) * w[:, None]
    Tn = np.moveaxis(T, n, -1)                     # fibres along mode n
    Y = Tn[tuple(samples[:, j] for j in range(len(others)))] * w[:, None]
    return Z, Y, samples, w


def fibre_rows_coo(idx: np.ndarray, vals: np.ndarray, dims, n: int, samples: np.ndarray,
                   w: np.ndarray) -> np.ndarray:
    """Sampled rows of the unfolding of a COO tensor: Y = S T_(n)^T for a sampling
    sketch S whose row j picks column (sample j) of T_(n) with weight w_j (Sec. 3.2,
    importance-sampling definition).  Row j is w_j times the mode-n fibre of T at the
    sampled multi-index: the values of the nonzeros whose other coordinates equal it,
    added at their mode-n coordinate (repeated coordinates add).  The cost is the
    paper's O(m s) gather once the nonzeros are grouped by fibre (here by a sort)."""
    N = len(dims)
    others = [k for k in range(N) if k != n]
    odims = [int(dims[k]) for k in others]
    col = np.ravel_multi_index(tuple(idx[k].astype(np.int64) for k in others), odims)
    key = np.ravel_multi_index(tuple(samples[:, j].astype(np.int64) for j in range(len(others))),
                               odims)
    order = np.argsort(col, kind="stable")
    sc = col[order]
    Y = np.zeros((samples.shape[0], int(dims[n])))
    for j in range(samples.shape[0]):
        lo = np.searchsorted(sc, key[j], side="left")
        hi = np.searchsorted(sc, key[j], side="right")
        e = order[lo:hi]
        np.add.at(Y[j], idx[n, e].astype(np.int64), vals[e].astype(np.float64))
        Y[j] *= w[j]
    return Y


def leverage_sketch_coo(idx, vals, dims, n: int, factors, m: int, seed: int, sweep: int):
    """leverage_sketch_dense for a COO tensor: the same draws and Z; Y gathered from
    the nonzeros of the sampled fibres (fibre_rows_coo)."""
    others = [k for k in range(len(dims)) if k != n]
    samples, w = leverage_draws(dims, n, factors, m, seed, sweep)
    Z = kron_rows(factors, others, samples) * w[:, None]
    return Z, fibre_rows_coo(idx, vals, dims, n, samples, w), samples, w


def leverage_sketch_coo_det(idx, vals, dims, n: int, factors, m: int):
    """leverage_sketch_dense_det for a COO tensor (unit weights)."""
    others = [k for k in range(len(dims)) if k != n]
    lin = leverage_select_det([leverage_scores(factors[k]) for k in others], m)
    samples = np.stack(np.unravel_index(lin, [int(dims[k]) for k in others]), axis=1)
    Z = kron_rows(factors, others, samples)
    return Z, fibre_rows_coo(idx, vals, dims, n, samples, np.ones(lin.shape[0])), samples
