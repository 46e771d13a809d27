"""Pins of the oracle's solves (Sec. 4, Alg. 5) and drivers (Algs. 1-4, 6)."""

import numpy as np
import pytest

from oracle import rng, sketch, solve, tucker
from oracle.tensor import kron_chain, reconstruct, unfold
from paper_2104_01101_gb300 import synth


# ---------------------------------------------------------------- solves

def _problem(seed, m=60, r=8, s=30, R=3, noise=0.0):
    g = np.random.default_rng(seed)
    Z = g.standard_normal((m, r))
    X0 = g.standard_normal((r, R)) @ g.standard_normal((R, s))
    Y = Z @ X0 + noise * g.standard_normal((m, s))
    return Z, Y, X0


def test_exact_solve_is_truncated_lstsq_and_optimal():
    Z, Y, _ = _problem(0, noise=0.5)
    R = 3
    Cn, V = solve.lrls_exact(Z, Y, R)
    B = Cn @ V.T
    assert np.allclose(V.T @ V, np.eye(R), atol=1e-12)
    X = np.linalg.solve(Z.T @ Z, Z.T @ Y)                # closed-form normal equations
    sig = np.linalg.svd(X, compute_uv=False)
    # Eckart-Young: ||X - B||^2 = sum of the discarded sigma^2
    assert np.sum((X - B) ** 2) == pytest.approx(np.sum(sig[R:] ** 2), rel=1e-10)
    # Pythagorean split of the residual (Appendix A): ||ZB - Y||^2 = ||ZX - Y||^2 + ||Z(X - B)||^2
    lhs = np.sum((Z @ B - Y) ** 2)
    rhs = np.sum((Z @ X - Y) ** 2) + np.sum((Z @ (X - B)) ** 2)
    assert lhs == pytest.approx(rhs, rel=1e-10)


def test_exact_solve_beats_random_rank_r_candidates_when_Z_orthonormal():
    g = np.random.default_rng(1)
    Z = np.linalg.qr(g.standard_normal((40, 6)))[0]
    Y = g.standard_normal((40, 12))
    Cn, V = solve.lrls_exact(Z, Y, 2)
    best = np.sum((Z @ Cn @ V.T - Y) ** 2)
    for _ in range(200):
        B = g.standard_normal((6, 2)) @ g.standard_normal((2, 12))
        assert np.sum((Z @ B - Y) ** 2) >= best - 1e-12


def test_rsvd_equals_exact_when_rank_fits_the_test_matrix():
    Z, Y, _ = _problem(2, noise=0.0)
    R, k = 3, 5
    Om = np.random.default_rng(9).standard_normal((Y.shape[1], k))
    Ce, Ve = solve.lrls_exact(Z, Y, R)
    Cr, Vr = solve.rsvd_lrls(Z, Y, R, Om)
    assert np.allclose(Ve, Vr, atol=1e-10) and np.allclose(Ce, Cr, atol=1e-9)


def test_rsvd_with_full_width_test_matrix_equals_exact():
    Z, Y, _ = _problem(3, noise=1.0)
    R = 3
    Om = np.random.default_rng(1).standard_normal((Y.shape[1], Z.shape[1]))
    Ce, Ve = solve.lrls_exact(Z, Y, R)
    Cr, Vr = solve.rsvd_lrls(Z, Y, R, Om)
    assert np.allclose(Ce @ Ve.T, Cr @ Vr.T, atol=1e-9)


def test_canonical_signs():
    g = np.random.default_rng(4)
    Cn, V = g.standard_normal((5, 3)), g.standard_normal((9, 3))
    C2, V2 = solve.canonical_signs(Cn, V)
    assert np.allclose(C2 @ V2.T, Cn @ V.T)
    idx = np.argmax(np.abs(V2), axis=0)
    assert np.all(V2[idx, np.arange(3)] > 0)


# ---------------------------------------------------------------- conventions and fitness

def test_unfolding_matches_kronecker_convention():
    g = np.random.default_rng(5)
    dims, ranks = (5, 4, 6), (2, 3, 2)
    core = g.standard_normal(ranks)
    A = [g.standard_normal((s, R)) for s, R in zip(dims, ranks)]
    T = reconstruct(core, A)
    assert np.allclose(T, np.einsum("abc,ia,jb,kc->ijk", core, *A))
    for n in range(3):
        P = tucker.kron_P(A, n)
        assert np.allclose(unfold(T, n).T, P @ unfold(core, n).T @ A[n].T)


def test_coo_fitness_identity_matches_direct_reconstruction():
    g = np.random.default_rng(6)
    dims, ranks = (6, 5, 7), (2, 2, 3)
    nnz = 400
    idx = np.stack([g.integers(0, s, nnz) for s in dims])
    vals = g.standard_normal(nnz)
    dense = np.zeros(dims)
    np.add.at(dense, tuple(idx), vals)
    core = g.standard_normal(ranks)
    A = [np.linalg.qr(g.standard_normal((s, R)))[0] for s, R in zip(dims, ranks)]
    direct = np.linalg.norm(dense - reconstruct(core, A)) / np.linalg.norm(dense)
    assert tucker.residual(tucker.Coo(idx, vals, dims), core, A) == pytest.approx(direct, rel=1e-10)
    assert tucker.residual(dense, core, A) == pytest.approx(direct, rel=1e-12)
    # non-orthonormal factors: the norm term is still exact
    B = [a * 1.7 for a in A]
    direct = np.linalg.norm(dense - reconstruct(core, B)) / np.linalg.norm(dense)
    assert tucker.residual(tucker.Coo(idx, vals, dims), core, B) == pytest.approx(direct, rel=1e-10)


# ---------------------------------------------------------------- drivers

def test_hosvd_and_hooi_recover_exact_tucker_tensor():
    T, core, A = synth.dense_tucker((12, 10, 9), (3, 2, 3), 0.0, seed=1)
    c, f = tucker.hooi(T, (3, 2, 3), 2)
    assert tucker.residual(T, c, f) < 1e-12
    for n in range(3):
        assert np.allclose(f[n] @ f[n].T, A[n] @ A[n].T, atol=1e-12)


def test_rrf_recovers_range_of_noiseless_low_rank_unfolding():
    T, core, A = synth.dense_tucker((30, 25, 20), (4, 3, 5), 0.0, seed=2)
    for n in (1, 2):
        k1, k2 = tucker.rrf_sizes(T.shape, n, A[n].shape[1], 200)
        U = tucker.init_rrf(T, n, A[n].shape[1], k1, k2, seed=5)
        assert np.allclose(U @ U.T, A[n] @ A[n].T, atol=1e-10)
        assert np.allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-12)


def test_rrf_sizes_reading():
    # Sec. 7: RRF sketch size sqrt(K) R with m = K R^2  ->  sqrt(m)
    assert tucker.rrf_sizes((40, 40, 40), 1, 5, 400) == (20, 45)
    assert tucker.rrf_sizes((400, 400, 400), 1, 10, 2000, k1=15) == (15, 115)


def degenerate_tables(dims, n):
    """H_k(i) = i * prod_{l > k, l != n} s_l, S = +1: the TensorSketch becomes the identity."""
    others = [k for k in range(len(dims)) if k != n]
    tabs = []
    for j, k in enumerate(others):
        stride = int(np.prod([dims[l] for l in others[j + 1:]]))
        tabs.append((np.arange(dims[k]) * stride, np.ones(dims[k])))
    return tabs, int(np.prod([dims[k] for k in others]))


def test_identity_sketch_reduces_sketched_als_to_hooi():
    # With an identity TensorSketch, Z = P^(n) and Y = T_(n)^T: the exact sketched
    # subproblem is the HOOI update (eq. (Yn)), so both iterations coincide.
    dims, ranks = (7, 6, 5), (3, 2, 3)
    # the degenerate tables hash every multi-index to its own C-order position
    for n in range(3):
        t, mn = degenerate_tables(dims, n)
        H, S = sketch.ts_hash(t, mn)
        assert np.array_equal(H, np.arange(mn)) and np.all(S == 1)
    cube = (6, 6, 6)
    T, _, _ = synth.dense_tucker(cube, ranks, 0.3, seed=4)
    init = tucker.hosvd(T, ranks)
    tabs = {n: degenerate_tables(cube, n)[0] for n in range(3)}
    c_s, f_s, _ = tucker.sketch_tucker_als(T, ranks, 36, 3, seed=0, solve="exact",
                                           init_factors=init, ts_tables=tabs)
    c_h, f_h = tucker.hooi(T, ranks, 3, init=init)
    for n in range(3):
        assert np.allclose(f_s[n], f_h[n], atol=1e-12)
    assert np.allclose(c_s, c_h, atol=1e-12)


@pytest.mark.parametrize("kind", ["ts", "lev"])
def test_exact_recovery_of_noiseless_tucker_tensor(kind):
    T, _, _ = synth.dense_tucker((40, 40, 40), (5, 5, 5), 0.0, seed=5)
    _, _, fits = tucker.sketch_tucker_als(T, (5, 5, 5), 400, 1, seed=7, kind=kind, track_fit=True)
    assert fits[0] < 1e-10


@pytest.mark.parametrize("kind", ["ts", "lev"])
def test_noisy_small_dense_within_ten_percent_of_hooi(kind):
    T, _, _ = synth.dense_tucker((40, 40, 40), (5, 5, 5), 1e-3, seed=0)
    c, f, fits = tucker.sketch_tucker_als(T, (5, 5, 5), 400, 5, seed=1, kind=kind, track_fit=True)
    ch, fh = tucker.hooi(T, (5, 5, 5), 5)
    assert fits[-1] <= 1.1 * tucker.residual(T, ch, fh)


def test_coo_and_dense_sketched_als_agree():
    # The input sketch is linear in the entries, so a COO tensor and its dense
    # form produce the same sketches and the same iterates.
    g = np.random.default_rng(8)
    dims, ranks = (12, 11, 10), (3, 3, 2)
    T, _, _ = synth.dense_tucker(dims, ranks, 0.05, seed=8)
    flat = np.flatnonzero(g.random(T.size) < 0.7)
    idx = np.array(np.unravel_index(flat, dims))
    vals = T.reshape(-1)[flat]
    # split a few entries into duplicates
    idx = np.concatenate([idx, idx[:, :30]], axis=1)
    vals = np.concatenate([vals * 1.0, np.zeros(30)])
    vals[:30] *= 0.5
    vals[-30:] = vals[:30]
    dense = np.zeros(dims)
    np.add.at(dense, tuple(idx), vals)
    X = tucker.Coo(idx, vals, dims)
    c1, f1, r1 = tucker.sketch_tucker_als(X, ranks, 120, 2, seed=3, track_fit=True)
    c2, f2, r2 = tucker.sketch_tucker_als(dense, ranks, 120, 2, seed=3, track_fit=True)
    for n in range(3):
        assert np.allclose(f1[n], f2[n], atol=1e-10)
    assert np.allclose(r1, r2, rtol=1e-8)


def test_cp_als_and_cp_sketch_tucker_recover_exact_cp_tensor():
    g = np.random.default_rng(9)
    dims, R = (20, 18, 16), 3
    A = [g.standard_normal((s, R)) for s in dims]
    T = tucker.cp_reconstruct(A)
    assert np.allclose(T, np.einsum("ir,jr,kr->ijk", *A))
    kr = tucker.khatri_rao([A[1], A[2]])
    assert np.allclose(kr, np.stack([np.kron(A[1][:, r], A[2][:, r]) for r in range(R)], 1))
    B, core, Bt, Ac = tucker.cp_sketch_tucker(T, R, (4, 4, 4), 200, 3, 60, seed=2)
    rel = np.linalg.norm(T - tucker.cp_reconstruct(B)) / np.linalg.norm(T)
    assert rel < 1e-6
