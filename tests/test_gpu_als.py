"""End-to-end parity of Sketch-Tucker-ALS (Alg. 4) on the GPU against the FP64 oracle."""

import numpy as np
import pytest
import torch

from oracle import tucker
from paper_2104_01101_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ts():
    from paper_2104_01101_gb300 import build, tsketch
    build.build_library()
    tsketch.lib()
    return tsketch


def proj(A):
    return A @ A.T


@pytest.mark.parametrize("kind,solve", [("ts", "rsvd"), ("ts", "exact"), ("lev", "rsvd"),
                                        ("lev", "exact"), ("lev_det", "rsvd"),
                                        ("lev_det", "exact")])
def test_small_dense_fp64_matches_oracle(ts, kind, solve):
    # 40^3 FP64, Tucker rank 5 plus 1e-3 noise, m = 400, 5 sweeps, RRF init
    dims, ranks, m, sweeps, seed = (40, 40, 40), (5, 5, 5), 400, 5, 1
    T, _, _ = synth.dense_tucker(dims, ranks, 1e-3, seed=0)
    k = {"ts": ts.TENSORSKETCH, "lev": ts.LEVERAGE, "lev_det": ts.LEVERAGE_DET}[kind]
    s = ts.SOLVE_RSVD if solve == "rsvd" else ts.SOLVE_EXACT
    core, fac, res = ts.tucker_als_sketched(torch.from_numpy(T).cuda(), ranks, m, sweeps, kind=k,
                                            seed=seed, solve=s, track_fit=True)
    c_o, f_o, r_o = tucker.sketch_tucker_als(T, ranks, m, sweeps, seed=seed, kind=kind,
                                             solve=solve, track_fit=True)
    assert np.allclose(res.cpu().numpy(), r_o, rtol=1e-9, atol=0)
    for n in range(3):
        assert np.abs(proj(fac[n].cpu().numpy()) - proj(f_o[n])).max() < 1e-9
    Tg = tucker.reconstruct(core.cpu().numpy(), [f.cpu().numpy() for f in fac])
    To = tucker.reconstruct(c_o, f_o)
    assert np.linalg.norm(Tg - To) <= 1e-9 * np.linalg.norm(To)


@pytest.mark.parametrize("kind", ["ts", "lev", "lev_det"])
def test_tensor_with_large_coherence_fp64_matches_oracle(ts, kind):
    # Sec. 7's Tensor 4 at 40^3: rank-5 Tucker plus 10 large entries; the leverage
    # scores of the RRF-initialised factors concentrate on the spikes' rows.
    dims, ranks, m, sweeps, seed = (40, 40, 40), (5, 5, 5), 400, 5, 3
    T, _, _ = synth.spiked_tucker(dims, ranks, 1e-3, seed=2)
    k = {"ts": ts.TENSORSKETCH, "lev": ts.LEVERAGE, "lev_det": ts.LEVERAGE_DET}[kind]
    core, fac, res = ts.tucker_als_sketched(torch.from_numpy(T).cuda(), ranks, m, sweeps, kind=k,
                                            seed=seed, track_fit=True)
    c_o, f_o, r_o = tucker.sketch_tucker_als(T, ranks, m, sweeps, seed=seed, kind=kind,
                                             track_fit=True)
    assert np.allclose(res.cpu().numpy(), r_o, rtol=1e-9, atol=0)
    for n in range(3):
        assert np.abs(proj(fac[n].cpu().numpy()) - proj(f_o[n])).max() < 1e-9


@pytest.mark.parametrize("solve", ["rsvd", "exact"])
def test_tall_mode_matches_oracle(ts, solve):
    # s = 8000 in mode 1: its Init-RRF factor and its subproblem take the multi-block
    # finalize (column signs over 2048-row chunks, then the write), not the fused solve
    dims, ranks, m, sweeps, seed = (30, 8000, 20), (3, 3, 2), 200, 2, 5
    T, _, _ = synth.dense_tucker(dims, ranks, 1e-2, seed=6)
    s_kind = ts.SOLVE_RSVD if solve == "rsvd" else ts.SOLVE_EXACT
    core, fac, res = ts.tucker_als_sketched(torch.from_numpy(T).cuda(), ranks, m, sweeps,
                                            seed=seed, solve=s_kind, track_fit=True)
    c_o, f_o, r_o = tucker.sketch_tucker_als(T, ranks, m, sweeps, seed=seed, solve=solve,
                                             track_fit=True)
    assert np.allclose(res.cpu().numpy(), r_o, rtol=1e-9, atol=0)
    for n in range(3):
        # factors themselves (signs included), not only their projectors
        assert np.abs(fac[n].cpu().numpy() - f_o[n]).max() < 1e-9


def test_wide_mode_many_sweeps_matches_oracle(ts):
    # s = 20000 in mode 0 with 6 sweeps of k = 14 (oversampling 10): Y_0 Omega for all
    # sweeps (84 columns) takes the split product over s in two column groups of <= 80
    dims, ranks, m, sweeps, seed = (20000, 20, 20), (4, 4, 4), 256, 6, 2
    T, _, _ = synth.dense_tucker(dims, ranks, 1e-2, seed=12)
    core, fac, res = ts.tucker_als_sketched(torch.from_numpy(T).cuda(), ranks, m, sweeps,
                                            seed=seed, oversample=10)
    c_o, f_o, _ = tucker.sketch_tucker_als(T, ranks, m, sweeps, seed=seed, oversample=10)
    r_o = tucker.residual(T, c_o, f_o)
    assert abs(float(res[0]) - r_o) <= 1e-9 * r_o
    for n in range(3):
        assert np.abs(proj(fac[n].cpu().numpy()) - proj(f_o[n])).max() < 1e-9


@pytest.mark.parametrize("kind", ["ts", "lev"])
def test_exact_recovery_noiseless(ts, kind):
    T, _, _ = synth.dense_tucker((40, 40, 40), (5, 5, 5), 0.0, seed=2)
    k = ts.TENSORSKETCH if kind == "ts" else ts.LEVERAGE
    _, _, res = ts.tucker_als_sketched(torch.from_numpy(T).cuda(), (5, 5, 5), 400, 1, kind=k,
                                       seed=4, track_fit=True)
    assert float(res[0]) < 1e-10


def test_identity_sketch_equals_hooi_on_gpu(ts):
    # Identity TensorSketch (degenerate tables, S = +1, m = s^2) with the exact solve
    # reproduces HOOI from the same initial factors.
    dims, ranks = (6, 6, 6), (3, 2, 3)
    T, _, _ = synth.dense_tucker(dims, ranks, 0.3, seed=4)
    init = tucker.hosvd(T, ranks)
    Tg = torch.from_numpy(T).cuda()
    m = 36
    # Drive the subproblem solve directly with the identity sketch (Z = P, Y = T_(n)^T).
    A = [torch.from_numpy(a).cuda() for a in init]
    c_h, f_h = tucker.hooi(T, ranks, 3, init=init)
    for sweep in range(3):
        for n in range(3):
            others = [k for k in range(3) if k != n]
            tabs = []
            for j, k in enumerate(others):
                stride = int(np.prod([dims[l] for l in others[j + 1:]]))
                tabs.append(torch.from_numpy((np.arange(dims[k]) * stride).astype(np.int32)).cuda())
            Z = ts.tensorsketch_apply([A[k] for k in others], tabs, m)
            Y = ts.tensorsketch_input(Tg, n, [tabs[others.index(k)] if k in others else None
                                              for k in range(3)], m)
            _, An = ts.lrls_solve(Z, Y, ranks[n], ts.SOLVE_EXACT)
            A[n] = An
    for n in range(3):
        assert np.abs(A[n].cpu().numpy() - f_h[n]).max() < 1e-10


def test_medium_dense_fp32_matches_oracle(ts):
    # 120^3 FP32 with the 400^3 workload's structure (decaying core, rank 10, noise 1e-2)
    dims, ranks, m, sweeps, seed = (120, 120, 120), (10, 10, 10), 2000, 3, 5
    T, _, _ = synth.dense_tucker(dims, ranks, 1e-2, seed=3, core_decay=0.9, dtype=np.float32)
    core, fac, res = ts.tucker_als_sketched(torch.from_numpy(T).cuda(), ranks, m, sweeps,
                                            seed=seed, rrf_k1=15, track_fit=True)
    _, f_o, r_o = tucker.sketch_tucker_als(T.astype(np.float64), ranks, m, sweeps, seed=seed,
                                           rrf_k1=15, track_fit=True)
    assert np.allclose(res.cpu().numpy(), r_o, rtol=1e-5, atol=0)
    for n in range(3):
        assert np.abs(proj(fac[n].double().cpu().numpy()) - proj(f_o[n])).max() < 1e-4


@pytest.fixture(scope="module")
def full_size_workload():
    # The benchmark workload itself: 400^3 FP32, rank 10, decaying core, noise 1e-2,
    # m = 2000, RRF k1 = 15, 10 sweeps; the FP64 oracle's decomposition of it.
    dims, ranks, m, sweeps, seed = (400, 400, 400), (10, 10, 10), 2000, 10, 7
    T, _, _ = synth.dense_tucker(dims, ranks, 1e-2, seed=1, core_decay=0.9, dtype=np.float32)
    T64 = T.astype(np.float64)
    c_o, f_o, _ = tucker.sketch_tucker_als(T64, ranks, m, sweeps, seed=seed, rrf_k1=15)
    r_final = tucker.residual(T64, c_o, f_o)
    return T, (ranks, m, sweeps, seed), f_o, r_final


@pytest.mark.parametrize("fp64", [False, True], ids=["fp32-solve", "fp64-qr-svd"])
def test_full_size_fp32_workload_matches_oracle(ts, full_size_workload, fp64):
    T, (ranks, m, sweeps, seed), f_o, r_final = full_size_workload
    core, fac, res = ts.tucker_als_sketched(torch.from_numpy(T).cuda(), ranks, m, sweeps,
                                            seed=seed, rrf_k1=15, solve_fp64=fp64)
    assert abs(float(res[0]) - r_final) <= 1e-5 * r_final
    for n in range(3):
        assert np.abs(proj(fac[n].double().cpu().numpy()) - proj(f_o[n])).max() < 1e-4


@pytest.mark.parametrize("fp64", [False, True], ids=["fp32-solve", "fp64-qr-svd"])
def test_full_size_bf16_workload_matches_oracle(ts, full_size_workload, fp64):
    # The precision form on the benchmark workload: every subproblem's Gram products in
    # BF16 on the tensor cores (FP32 accumulation), the QR and SVD of the small system in
    # FP32 or FP64, against the FP64 oracle: BF16 stages are held to 1e-2 relative, the
    # residual also to 1e-3 absolute (the equal-residual criterion), the factors'
    # projectors to 1e-2.
    T, (ranks, m, sweeps, seed), f_o, r_final = full_size_workload
    core, fac, res = ts.tucker_als_sketched(torch.from_numpy(T).cuda(), ranks, m, sweeps,
                                            seed=seed, rrf_k1=15, gram_bf16=True,
                                            solve_fp64=fp64)
    r = float(res[0])
    assert abs(r - r_final) <= 1e-2 * r_final and abs(r - r_final) <= 1e-3
    for n in range(3):
        assert np.abs(proj(fac[n].double().cpu().numpy()) - proj(f_o[n])).max() < 1e-2


def test_non_finite_input_raises_numeric_error(ts):
    # A NaN in the data reaches the Gram matrices of the sketched subproblems; the solve
    # flags it on the device and the call reports TS_ERR_NUMERIC (status 6).
    T, _, _ = synth.dense_tucker((40, 40, 40), (5, 5, 5), 1e-3, seed=0)
    T[3, 7, 11] = np.nan
    with pytest.raises(ts.TsError) as e:
        ts.tucker_als_sketched(torch.from_numpy(T).cuda(), (5, 5, 5), 400, 2, seed=1)
    assert e.value.status == 6


def test_medium_dense_fp32_with_fp64_solve_matches_oracle(ts):
    # precision form of the small solve: FP64 QR and final FP64 Jacobi sweeps on FP32 data
    dims, ranks, m, sweeps, seed = (120, 120, 120), (10, 10, 10), 2000, 3, 5
    T, _, _ = synth.dense_tucker(dims, ranks, 1e-2, seed=3, core_decay=0.9, dtype=np.float32)
    core, fac, res = ts.tucker_als_sketched(torch.from_numpy(T).cuda(), ranks, m, sweeps,
                                            seed=seed, rrf_k1=15, track_fit=True, solve_fp64=True)
    _, f_o, r_o = tucker.sketch_tucker_als(T.astype(np.float64), ranks, m, sweeps, seed=seed,
                                           rrf_k1=15, track_fit=True)
    assert np.allclose(res.cpu().numpy(), r_o, rtol=1e-5, atol=0)
    for n in range(3):
        assert np.abs(proj(fac[n].double().cpu().numpy()) - proj(f_o[n])).max() < 1e-4


@pytest.mark.parametrize("solve", ["rsvd", "exact"])
def test_medium_dense_bf16_gram_form_matches_oracle(ts, solve):
    # precision form: every subproblem's [Z^T Z | Z^T Y Omega | Z^T Y] in BF16 on the tensor
    # cores with FP32 accumulation.  BF16 stages are held to 1e-2 (relative) against the
    # FP64 oracle, and the residual to 1e-3 absolute, the equal-residual criterion.
    dims, ranks, m, sweeps, seed = (120, 120, 120), (10, 10, 10), 2000, 3, 5
    kind = ts.SOLVE_RSVD if solve == "rsvd" else ts.SOLVE_EXACT
    if solve == "exact":
        ranks, m = (5, 5, 5), 400
    T, _, _ = synth.dense_tucker(dims, ranks, 1e-2, seed=3, core_decay=0.9, dtype=np.float32)
    core, fac, res = ts.tucker_als_sketched(torch.from_numpy(T).cuda(), ranks, m, sweeps,
                                            seed=seed, rrf_k1=15, track_fit=True, solve=kind,
                                            gram_bf16=True)
    _, f_o, r_o = tucker.sketch_tucker_als(T.astype(np.float64), ranks, m, sweeps, seed=seed,
                                           rrf_k1=15, track_fit=True,
                                           solve="rsvd" if solve == "rsvd" else "exact")
    res, r_o = res.cpu().numpy(), np.asarray(r_o)
    assert np.all(np.abs(res - r_o) <= 1e-2 * r_o)
    assert np.all(np.abs(res - r_o) <= 1e-3)
    for n in range(3):
        assert np.abs(proj(fac[n].double().cpu().numpy()) - proj(f_o[n])).max() < 1e-2


def test_graph_replay_matches_direct_enqueue(ts):
    # use_graph captures the decomposition once and replays it; replays must read the
    # current contents of the caller's buffers (here the tensor is rescaled in place).
    dims, ranks, m = (120, 120, 120), (10, 10, 10), 2000
    T, _, _ = synth.dense_tucker(dims, ranks, 1e-2, seed=3, core_decay=0.9, dtype=np.float32)
    X = torch.from_numpy(T).cuda()
    direct = ts.TuckerPlan(X, ranks, m, 3, seed=2, rrf_k1=15).run(X)
    graph = ts.TuckerPlan(X, ranks, m, 3, seed=2, rrf_k1=15, use_graph=True)
    graph.run(X)
    graph.run(X)
    torch.cuda.synchronize()
    r_d, r_g = float(direct.residuals[0]), float(graph.residuals[0])
    assert abs(r_d - r_g) <= 1e-5 * r_d
    core_before = graph.core.clone()
    X.mul_(2.0)
    graph.run(X)
    torch.cuda.synchronize()
    assert abs(float(graph.residuals[0]) - r_d) <= 1e-5 * r_d
    assert torch.allclose(graph.core, 2.0 * core_before, rtol=1e-4, atol=1e-4)


def test_large_core_rank_uses_newton_schulz_and_matches_oracle(ts):
    # Tucker rank (20,20,20): r = 400 per subproblem, beyond the on-chip solve
    dims, ranks, m = (80, 80, 80), (20, 20, 20), 3000
    T, _, _ = synth.dense_tucker(dims, ranks, 1e-2, seed=7, dtype=np.float32)
    _, fac, res = ts.tucker_als_sketched(torch.from_numpy(T).cuda(), ranks, m, 2, seed=4,
                                         track_fit=True)
    _, f_o, r_o = tucker.sketch_tucker_als(T.astype(np.float64), ranks, m, 2, seed=4,
                                           track_fit=True)
    assert np.allclose(res.cpu().numpy(), r_o, rtol=1e-4, atol=0)
    for n in range(3):
        assert np.abs(proj(fac[n].double().cpu().numpy()) - proj(f_o[n])).max() < 1e-3


def test_order4_and_resketch(ts):
    dims, ranks, m = (20, 18, 16, 14), (3, 3, 2, 2), 300
    T, _, _ = synth.dense_tucker(dims, ranks, 1e-2, seed=6)
    core, fac, res = ts.tucker_als_sketched(torch.from_numpy(T).cuda(), ranks, m, 3, seed=3,
                                            resketch=True, track_fit=True)
    _, f_o, r_o = tucker.sketch_tucker_als(T, ranks, m, 3, seed=3, resketch=True, track_fit=True)
    assert np.allclose(res.cpu().numpy(), r_o, rtol=1e-9)


def test_coo_tensor_matches_oracle(ts):
    dims, ranks, m = (300, 250, 200), (4, 4, 4), 400
    idx, vals, _, _ = synth.coo_zipf_tucker(dims, 60000, ranks, seed=5, val_dtype=np.float64)
    X = ts.Coo(torch.from_numpy(idx).cuda(), torch.from_numpy(vals).cuda(), dims)
    core, fac, res = ts.tucker_als_sketched(X, ranks, m, 2, seed=8, track_fit=True)
    Xo = tucker.Coo(idx.astype(np.int64), vals, dims)
    c_o, f_o, r_o = tucker.sketch_tucker_als(Xo, ranks, m, 2, seed=8, track_fit=True)
    for n in range(3):
        assert np.abs(proj(fac[n].cpu().numpy()) - proj(f_o[n])).max() < 1e-9
    # COO residuals on the device (repeated coordinates merged) after every sweep
    assert np.allclose(res.cpu().numpy(), r_o, rtol=1e-9, atol=0)


@pytest.mark.parametrize("kind", ["lev", "lev_det"])
@pytest.mark.parametrize("dtype", [torch.float64])
def test_coo_leverage_als_matches_oracle(ts, kind, dtype):
    # Leverage sampling of a COO tensor (fibre index on the device) against the
    # oracle's COO run (FP64: the draws and the selection follow the factor bits, so
    # FP32 runs may pick other rows; the FP32 sketch is checked on its own).
    dims, ranks, m, sweeps, seed = (30, 25, 20), (3, 3, 2), 60, 3, 4
    npd = np.float64 if dtype == torch.float64 else np.float32
    idx, vals, _, _ = synth.coo_zipf_tucker(dims, 4000, ranks, seed=3, val_dtype=npd)
    X = ts.Coo(torch.from_numpy(idx).cuda().contiguous(), torch.from_numpy(vals).cuda(), dims)
    k = ts.LEVERAGE if kind == "lev" else ts.LEVERAGE_DET
    core, fac, _ = ts.tucker_als_sketched(X, ranks, m, sweeps, kind=k, seed=seed,
                                          want_residual=False)
    Xo = tucker.Coo(idx, vals.astype(np.float64), dims)
    c_o, f_o, _ = tucker.sketch_tucker_als(Xo, ranks, m, sweeps, seed=seed, kind=kind)
    Tg = tucker.reconstruct(core.double().cpu().numpy(), [f.double().cpu().numpy() for f in fac])
    To = tucker.reconstruct(c_o, f_o)
    tol = 1e-9 if dtype == torch.float64 else 2e-3
    assert np.linalg.norm(Tg - To) <= tol * np.linalg.norm(To)


def test_shape_errors(ts):
    T = torch.zeros((10, 10, 10), dtype=torch.float64, device="cuda")
    with pytest.raises(ts.TsError) as e:
        ts.tucker_als_sketched(T, (10, 2, 2), 50, 1)
    assert e.value.status == 2
    with pytest.raises(ts.TsError) as e:
        ts.tucker_als_sketched(T, (3, 3, 3), 8, 1)     # m < 9
    assert e.value.status == 2


def test_cp_via_tucker_fp64_matches_oracle(ts):
    # Alg. 6 on a small collinear CP tensor: Tucker (6,6,6) then CP-ALS rank 4 on the core
    T, _ = synth.cp_collinear((30, 28, 26), 4, 0.5, 1e-3, seed=2)
    outs, res = ts.cp_via_tucker(torch.from_numpy(T).cuda(), 4, (6, 6, 6), 300, 3, 10, seed=3)
    B, core, Bt, Ac = tucker.cp_sketch_tucker(T, 4, (6, 6, 6), 300, 3, 10, seed=3)
    # CP-ALS normal equations amplify rounding by cond(Gamma) per sweep (collinear factors)
    for k in range(3):
        assert np.abs(outs[k].cpu().numpy() - B[k]).max() <= 1e-6 * np.abs(B[k]).max()
    want = np.linalg.norm(T - tucker.cp_reconstruct(B)) / np.linalg.norm(T)
    assert abs(res - want) <= 1e-7 * max(want, 1e-12)


def test_cp_via_tucker_coo_residual(ts):
    # Alg. 6 on a COO copy of a small CP tensor (every entry once plus cancelling
    # repeats): the residual on the device equals the oracle's COO identity on the
    # returned factors and the dense residual of the same factors.
    T, _ = synth.cp_collinear((20, 18, 16), 3, 0.5, 1e-3, seed=5)
    dims = T.shape
    idx = np.stack(np.unravel_index(np.arange(T.size), dims)).astype(np.int32)
    vals = T.reshape(-1).copy()
    idx = np.concatenate([idx, idx[:, :40]], axis=1)
    vals = np.concatenate([vals, np.zeros(40)])
    vals[:40] -= 0.5
    vals[-40:] += 0.5
    X = ts.Coo(torch.from_numpy(idx).cuda().contiguous(), torch.from_numpy(vals).cuda(), dims)
    outs, res = ts.cp_via_tucker(X, 3, (5, 5, 5), 200, 3, 10, seed=3)
    B = [o.cpu().numpy() for o in outs]
    want = np.linalg.norm(T - tucker.cp_reconstruct(B)) / np.linalg.norm(T)
    assert abs(res - want) <= 1e-7 * max(want, 1e-9) + 1e-9


def _signal_projectors(core, factors, R_sig):
    """Projector onto the leading R_sig left singular vectors of A^(n) C_(n) for every
    mode: the part of a Tucker model's column spaces that carries the signal (gauge-free)."""
    out = []
    for n, A in enumerate(factors):
        U = np.linalg.svd(A @ tucker.unfold(core, n), full_matrices=False)[0][:, :R_sig]
        out.append(U @ U.T)
    return out


def _gram_condition(A):
    """max over modes of cond(*_{k != n} A_k^T A_k): the amplification of rounding in the
    normal equations of a CP-ALS update (Alg. 2)."""
    worst = 1.0
    for n in range(len(A)):
        G = np.ones((A[0].shape[1],) * 2)
        for k in range(len(A)):
            if k != n:
                G = G * (A[k].T @ A[k])
        worst = max(worst, np.linalg.cond(G))
    return worst


def _noise_energy_bound(core_g, core_o, R_cp, T64, res_g, res_o):
    """Relative residual difference that the noise directions allow.  With orthonormal
    factors res^2 ||T||^2 = ||T||^2 - ||core||^2; both decompositions hold the signal
    subspace, and the directions beyond the CP rank (noise) may capture any part of the
    noise energy.  So |res_g^2 - res_o^2| ||T||^2 is at most the energy that the
    trailing singular values (index >= R_cp) of each side's core unfoldings carry, and
    |res_g - res_o| / res_o at most that divided by (res_g + res_o) res_o ||T||^2."""
    e = 0.0
    for c in (core_g, core_o):
        for n in range(3):
            sv = np.linalg.svd(tucker.unfold(c, n), compute_uv=False)
            e += float(np.sum(sv[R_cp:] ** 2))
    return e / ((res_g + res_o) * res_o * float(np.sum(T64 ** 2)))


def _cp_stagewise(ts, T, R_cp, tranks, m, tsweeps, csweeps, seed):
    """cp_via_tucker (Alg. 6) on FP32 data, stage by stage against the FP64 oracle:
    (1) the sketched Tucker-ALS it starts from, (2) CP-ALS on the GPU's own Tucker core
    (the GPU's ts_cp_als and the oracle's cp_als from the same core and the same HOSVD
    start), (3) the whole call.  Returns the measured deviations and the bounds they are
    held to."""
    T64 = T.astype(np.float64)
    Tg = torch.from_numpy(T).cuda()
    core, fac, res = ts.tucker_als_sketched(Tg, tranks, m, tsweeps, seed=seed)
    c_o, f_o, _ = tucker.sketch_tucker_als(T64, tranks, m, tsweeps, seed=seed)
    r_o = tucker.residual(T64, c_o, f_o)
    fac64 = [f.double().cpu().numpy() for f in fac]
    core64 = core.double().cpu().numpy()
    Pg = _signal_projectors(core64, fac64, R_cp)
    Po = _signal_projectors(c_o, f_o, R_cp)
    out = {"tucker_res": abs(float(res[0]) - r_o) / r_o,
           "tucker_res_bound": _noise_energy_bound(core64, c_o, R_cp, T64, float(res[0]), r_o),
           "tucker_signal_proj": max(np.abs(Pg[n] - Po[n]).max() for n in range(3))}
    A_g = [a.double().cpu().numpy() for a in ts.cp_als(core, R_cp, csweeps)]
    A_o = tucker.cp_als(core64, R_cp, csweeps, tucker.cp_init_hosvd(core64, R_cp))
    Kg, Ko = tucker.cp_reconstruct(A_g), tucker.cp_reconstruct(A_o)
    out["cp_model"] = np.linalg.norm(Kg - Ko) / np.linalg.norm(Ko)
    out["cp_fit_core"] = abs(np.linalg.norm(core64 - Kg) - np.linalg.norm(core64 - Ko)) / \
        np.linalg.norm(core64)
    out["gram_condition"] = _gram_condition(A_o)
    outs, res_cp = ts.cp_via_tucker(Tg, R_cp, tranks, m, tsweeps, csweeps, seed=seed)
    got = np.linalg.norm(T64 - tucker.cp_reconstruct([o.double().cpu().numpy() for o in outs]))
    out["cp_res_self"] = abs(res_cp - got / np.linalg.norm(T64)) / res_cp
    print(out)
    return out


def test_cp_als_fp32_well_conditioned_core_matches_oracle(ts):
    # CP-ALS arithmetic (ts_cp_als: HOSVD start, Alg. 2 sweeps) in FP32 against the FP64
    # oracle from the same core: a rank-10 CP core of 12^3 with orthonormal factors and
    # weights 1 .. 0.3, plus noise 1e-3 (cond(Gamma) near 1, so FP32 rounding stays at
    # its own level)
    g = np.random.default_rng(5)
    A0 = [np.linalg.qr(g.standard_normal((12, 10)))[0] for _ in range(3)]
    A0[0] = A0[0] * np.linspace(1.0, 0.3, 10)[None, :]
    core = tucker.cp_reconstruct(A0) + 1e-3 * g.standard_normal((12, 12, 12))
    core32 = core.astype(np.float32)
    A_g = [a.double().cpu().numpy() for a in ts.cp_als(torch.from_numpy(core32).cuda(), 10, 25)]
    c64 = core32.astype(np.float64)
    A_o = tucker.cp_als(c64, 10, 25, tucker.cp_init_hosvd(c64, 10))
    Kg, Ko = tucker.cp_reconstruct(A_g), tucker.cp_reconstruct(A_o)
    assert np.linalg.norm(Kg - Ko) <= 1e-5 * np.linalg.norm(Ko)
    for k in range(3):  # same start and gauge: the factors themselves
        assert np.abs(A_g[k] - A_o[k]).max() <= 1e-5 * np.abs(A_o[k]).max()


def test_cp_via_tucker_fp32_collinear_workload(ts):
    # The collinear-CP workload scaled down: rank-10 CP with pairwise cosine 0.9, noise
    # 1e-2, 60^3, Tucker (12,12,12), m = 1500, 2 Tucker sweeps, 25 CP sweeps.
    T, _ = synth.cp_collinear((60, 60, 60), 10, 0.9, 1e-2, seed=4, dtype=np.float32)
    T64 = T.astype(np.float64)
    tranks, m = (12, 12, 12), 1500
    # The Tucker stage in FP64 on the GPU equals the oracle: the code path is exact.
    _, f64, r64 = ts.tucker_als_sketched(torch.from_numpy(T64).cuda(), tranks, m, 2, seed=1)
    c_o, f_o, _ = tucker.sketch_tucker_als(T64, tranks, m, 2, seed=1)
    r_o = tucker.residual(T64, c_o, f_o)
    assert abs(float(r64[0]) - r_o) <= 1e-9 * r_o
    for n in range(3):
        assert np.abs(proj(f64[n].cpu().numpy()) - proj(f_o[n])).max() < 1e-8
    # FP32: each mode's core unfolding has one dominant direction (singular value 1), nine
    # signal directions near 0.016 and, Tucker rank 12 exceeding the CP rank 10, two noise
    # directions near 0.001.  FP32 rounding relative to the dominant direction is ~60x
    # larger relative to the signal, so: the noise directions' projectors may differ by
    # O(0.1); the signal subspace (10 leading directions, gap 0.014) is held to 1e-2;
    # the residual, whose last digits the noise directions carry, to the energy those
    # directions hold (plus FP32 rounding).
    d = _cp_stagewise(ts, T, 10, tranks, m, 2, 25, seed=1)
    assert d["tucker_signal_proj"] <= 1e-2
    assert d["tucker_res"] <= d["tucker_res_bound"] + 1e-5
    # CP-ALS on factors of pairwise cosine 0.9: cond(Gamma) of the normal equations is
    # ~1e3 to 1e5 (measured), which turns FP32 rounding into trajectories that differ
    # pointwise (the arithmetic itself is pinned at 1e-5 on a well-conditioned core); the
    # fits of the CP models to the core agree to 5e-3 of the core's norm
    assert d["cp_fit_core"] <= 5e-3
    assert d["cp_res_self"] <= 1e-4


def test_cp_via_tucker_collinear_workload_full_size(ts):
    # The collinear-CP workload at its stated size: 300^3 CP rank 20 with pairwise cosine
    # 0.9 plus noise 1e-2, sketched Tucker (25,25,25) with m = 3000 (r = 625 per
    # subproblem: the Newton-Schulz path), 5 Tucker sweeps, CP-ALS rank 20 for 25 sweeps.
    T, _ = synth.cp_collinear((300, 300, 300), 20, 0.9, 1e-2, seed=4, dtype=np.float32)
    # The same structure as the scaled case (one dominant direction, 19 signal directions,
    # 5 noise directions per mode), held to the same bounds.
    d = _cp_stagewise(ts, T, 20, (25, 25, 25), 3000, 5, 25, seed=3)
    assert d["tucker_signal_proj"] <= 1e-2
    assert d["tucker_res"] <= d["tucker_res_bound"] + 1e-5
    # CP-ALS on factors of pairwise cosine 0.9: cond(Gamma) of the normal equations is
    # ~1e3 to 1e5 (measured), which turns FP32 rounding into trajectories that differ
    # pointwise (the arithmetic itself is pinned at 1e-5 on a well-conditioned core); the
    # fits of the CP models to the core agree to 5e-3 of the core's norm
    assert d["cp_fit_core"] <= 5e-3
    assert d["cp_res_self"] <= 1e-4


def test_sparse_order4_scaled_workload_matches_oracle(ts):
    # The sparse 4-way workload scaled down (its recipe at dims 2000, 1e6 nonzeros):
    # Zipf(1.1) coordinates with duplicates, planted rank-(8,8,8,8) Tucker component of the
    # noise's norm, m = 4096, RRF k1 = 64, k2 = 128, re-sketched every sweep.  r = 512 per
    # subproblem: the RSVD solve inverts Z^T Z by Newton-Schulz products.
    dims, ranks, m = (2000, 2000, 2000, 2000), (8, 8, 8, 8), 4096
    idx, vals, _, _ = synth.coo_zipf_tucker(dims, 1_000_000, ranks, seed=9, val_dtype=np.float64)
    X = ts.Coo(torch.from_numpy(idx).cuda(), torch.from_numpy(vals).cuda(), dims)
    core, fac, _ = ts.tucker_als_sketched(X, ranks, m, 2, seed=6, rrf_k1=64, rrf_k2=128,
                                          resketch=True, want_residual=False)
    c_o, f_o, _ = tucker.sketch_tucker_als(tucker.Coo(idx.astype(np.int64), vals, dims), ranks, m,
                                           2, seed=6, rrf_k1=64, rrf_k2=128, resketch=True)
    for n in range(4):
        assert np.abs(proj(fac[n].cpu().numpy()) - proj(f_o[n])).max() < 1e-8
    # the core in the gauge of the factors: C x_n A_n^T A_n' is gauge-invariant per mode
    Cg = core.cpu().numpy()
    for n in range(4):
        U = np.moveaxis(Cg, n, 0).reshape(ranks[n], -1)
        V = np.moveaxis(c_o, n, 0).reshape(ranks[n], -1)
        sg = np.linalg.svd(U, compute_uv=False)
        so = np.linalg.svd(V, compute_uv=False)
        assert np.allclose(sg, so, rtol=1e-8, atol=1e-10 * so[0])


def test_sparse_full_size_decomposition_properties(ts):
    # The sparse 4-way workload at the size the benchmark times (200000^4, 1e8 nonzeros,
    # m = 4096, rank 8, 5 sweeps): too large for the oracle, so checked by properties that
    # hold at any size: no breakdown, orthonormal factors, a residual that repeats to the
    # rounding of the FP32 atomics, and one well below 1 (the planted component is found).
    dims, ranks, nnz, m = (200000,) * 4, (8,) * 4, 100_000_000, 4096
    idx, vals = synth.coo_zipf_tucker_torch(dims, nnz, ranks, seed=11, device="cuda")
    X = ts.Coo(idx, vals, dims)
    plan = ts.TuckerPlan(X, ranks, m, 5, seed=3, rrf_k1=64, rrf_k2=128)
    plan.run(X)
    r1 = float(plan.residuals[0])
    assert plan.numeric_flag() == 0
    for A in plan.factors:
        G = (A.double().t() @ A.double()).cpu().numpy()
        assert np.abs(G - np.eye(G.shape[0])).max() < 1e-4
    plan.run(X)
    r2 = float(plan.residuals[0])
    assert 0.0 < r1 < 0.5 and abs(r1 - r2) <= 1e-4 * r1


def test_deterministic_leverage_all_rows_is_hooi_on_gpu(ts):
    # m = prod of the other mode sizes keeps every row: with the exact solve the sketched
    # ALS is HOOI from the same initial factors
    dims, ranks = (7, 6, 5), (3, 2, 2)
    T, _, _ = synth.dense_tucker(dims, ranks, 0.3, seed=3)
    init = tucker.hosvd(T, ranks)
    m = 42
    Tg = torch.from_numpy(T).cuda()
    plan = ts.TuckerPlan(Tg, ranks, m, 3, kind=ts.LEVERAGE_DET, solve=ts.SOLVE_EXACT)
    plan.run(Tg, init_factors=[None] + [torch.from_numpy(a).cuda() for a in init[1:]])
    torch.cuda.synchronize()
    _, f_h = tucker.hooi(T, ranks, 3, init=init)
    for n in range(3):
        f = plan.factors[n].cpu().numpy()
        assert np.abs(f @ f.T - f_h[n] @ f_h[n].T).max() < 1e-10
