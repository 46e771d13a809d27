"""Float32 emulation of the FP32 forms' Q = qr(C) (Alg. 5, step "Q = qr(C)"): shifted
CholeskyQR3 (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa, SIAM J. Sci. Comput. 42,
2020) with the constants the cluster solve uses: the first pass factors C^T C + s I with
s = 11 (r k + k (k + 1)) 2^-24 ||C||_F^2, the unshifted passes drop a direction whose
pivot is not above 2^-40 tr / k, and the last pass is taken to first order when its Gram
is within 2^-12 of I.  The checks pin the design (orthogonality, span, dropped
directions), not the kernel's bits: the GPU parity tests compare the solve itself with
the oracle.  CPU only; no part of the library is imported.
"""
import numpy as np
import pytest

F32 = np.float32
KCK = 16


def _factor(S, r, k, mode):
    """N (unit lower, the inverse of L) and D^{-1/2} of S (+ shift) = L D L^T, in float32."""
    v = np.zeros((KCK, KCK), F32)
    v[:k, :k] = S[:k, :k]
    tr = F32(np.trace(v))
    if mode == 2 and np.all(np.abs(v[:k, :k] - np.eye(k, dtype=F32)) <= F32(2.0 ** -12)):
        dq = np.zeros(KCK, F32)
        dq[:k] = F32(1.5) - F32(0.5) * np.diag(v)[:k]
        N = np.eye(KCK, dtype=F32)
        low = np.tril_indices(KCK, -1)
        N[low] = -v[low]
        return N, dq
    thr = F32(2.0 ** -40) * tr / F32(k)
    if mode == 0:
        thr = F32(0)
        sh = F32(11 * (r * k + k * (k + 1))) * F32(2.0 ** -24) * tr
        v[np.arange(k), np.arange(k)] += sh
    dinv = np.zeros(KCK, F32)
    for j in range(KCK):
        d = v[j, j]
        dj = F32(1) / d if d > thr else F32(0)
        dinv[j] = dj
        row = v[j].copy()
        for i in range(j + 1, KCK):
            m = F32(v[i, j] * dj)
            upd = (v[i] - m * row).astype(F32)
            upd[j] = -m
            v[i] = upd
    N = np.where(np.tril(np.ones((KCK, KCK), bool), -1), v, F32(0))
    np.fill_diagonal(N, F32(1))
    return N, np.sqrt(dinv).astype(F32)


def cholqr3_f32(C, k):
    r = C.shape[0]
    X = np.zeros((r, KCK), F32)
    X[:, :C.shape[1]] = C
    for mode in (0, 1, 2):
        X[:, k:] = 0
        S = (X.T @ X).astype(F32)
        N, dq = _factor(S, r, k, mode)
        X = ((X @ N.T) * dq).astype(F32)
    X[:, k:] = 0
    return X.astype(np.float64)


def _conditioned(rng, r, k, kappa):
    U, _ = np.linalg.qr(rng.standard_normal((r, k)))
    V, _ = np.linalg.qr(rng.standard_normal((k, k)))
    return (U * np.logspace(0, -np.log10(kappa), k)) @ V.T


def _span_residual(Q, C):
    P = Q @ np.linalg.pinv(Q)
    return np.linalg.norm(C - P @ C) / np.linalg.norm(C)


@pytest.mark.parametrize("kappa", [1.0, 1e2, 1e4])
def test_orthonormal_basis_of_range(kappa):
    rng = np.random.default_rng(11)
    r, k = 100, 15
    C = _conditioned(rng, r, k, kappa)
    Q = cholqr3_f32(C, k)
    assert np.abs(Q[:, :k].T @ Q[:, :k] - np.eye(k)).max() < 1e-6
    assert _span_residual(Q[:, :k], C) < 1e-6


@pytest.mark.parametrize("seed", [11, 1])
def test_condition_near_float32_limit(seed):
    # kappa = 1e6: directions of C near 1e-6 sigma_1 (16 unit roundoffs) may be dropped;
    # what is kept stays orthonormal, and the span misses at most their energy
    rng = np.random.default_rng(seed)
    r, k = 100, 15
    C = _conditioned(rng, r, k, 1e6)
    Q = cholqr3_f32(C, k)[:, :k]
    kept = np.linalg.norm(Q, axis=0) > 0
    assert kept.sum() >= 11
    Qk = Q[:, kept]
    assert np.abs(Qk.T @ Qk - np.eye(kept.sum())).max() < 1e-5
    assert _span_residual(Qk, C) < 1e-4


def test_rank_deficient_columns_dropped_or_orthonormal():
    rng = np.random.default_rng(12)
    r, k = 100, 15
    C = rng.standard_normal((r, 10)) @ rng.standard_normal((10, k))
    Q = cholqr3_f32(C, k)[:, :k]
    norms = np.linalg.norm(Q, axis=0)
    kept = norms > 0
    assert kept.sum() >= 10
    assert np.allclose(norms[kept], 1.0, atol=1e-6)
    Qk = Q[:, kept]
    assert np.abs(Qk.T @ Qk - np.eye(kept.sum())).max() < 1e-5
    assert _span_residual(Qk, C) < 1e-6


def test_zero_columns_and_width_below_sixteen():
    rng = np.random.default_rng(13)
    r, k = 100, 15
    C = rng.standard_normal((r, k))
    C[:, 3] = 0
    C[:, 9] = 0
    Q = cholqr3_f32(C, k)
    norms = np.linalg.norm(Q, axis=0)
    assert norms[3] == 0 and norms[9] == 0 and norms[15] == 0
    assert np.allclose(np.delete(norms[:k], [3, 9]), 1.0, atol=1e-6)
    Q12 = cholqr3_f32(rng.standard_normal((r, 12)), 12)
    assert np.all(Q12[:, 12:] == 0)
    assert np.abs(Q12[:, :12].T @ Q12[:, :12] - np.eye(12)).max() < 1e-6


def test_zero_matrix_gives_zero_basis():
    Q = cholqr3_f32(np.zeros((40, 8)), 8)
    assert np.all(Q == 0)
