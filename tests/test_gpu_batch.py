"""Batched Sketch-Tucker-ALS (Alg. 4 on many tensors per launch) on the GPU: every
tensor of a batch equals its own decomposition by the FP64 oracle (FP64 data) and by
the single-tensor GPU driver with the same seed (FP32 data)."""

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


def batch_case(count, seed, dtype, lo=24, hi=72, rlo=3, rhi=7):
    # uneven shapes and ranks, one rank R per tensor, m = 8 R^2, noise 1e-2
    g = np.random.default_rng(seed)
    tensors, ranks, ms = [], [], []
    for i in range(count):
        dims = tuple(int(x) for x in g.integers(lo, hi + 1, size=3))
        R = int(g.integers(rlo, rhi + 1))
        T, _, _ = synth.dense_tucker(dims, (R, R, R), 1e-2, seed=1000 * seed + i, dtype=dtype)
        tensors.append(T)
        ranks.append((R, R, R))
        ms.append(8 * R * R)
    return tensors, ranks, ms


def test_batch_fp64_matches_oracle(ts):
    tensors, ranks, ms = batch_case(5, 1, np.float64)
    sweeps, seed = 3, 40
    b = ts.TuckerBatch([torch.from_numpy(T).cuda() for T in tensors], ranks, ms, sweeps,
                       seed=seed)
    b.sweeps()
    res = b.residual().cpu().numpy()
    assert b.flags() == [0] * len(tensors)
    for i, T in enumerate(tensors):
        c_o, f_o, _ = tucker.sketch_tucker_als(T, ranks[i], ms[i], sweeps, seed=seed + i)
        r_o = tucker.residual(T, c_o, f_o)
        assert abs(res[i] - r_o) <= 1e-9 * r_o
        for n in range(3):
            assert np.abs(proj(b.factors[i][n].cpu().numpy()) - proj(f_o[n])).max() < 1e-9
    b.close()


def test_batch_fp32_equals_single_tensor_driver(ts):
    tensors, ranks, ms = batch_case(8, 2, np.float32, hi=96, rhi=9)
    sweeps, seed = 4, 7
    Tg = [torch.from_numpy(T).cuda() for T in tensors]
    b = ts.TuckerBatch(Tg, ranks, ms, sweeps, seed=seed)
    b.sweeps()
    res = b.residual().cpu().numpy()
    assert b.flags() == [0] * len(tensors)
    tiles, times = b.tiles()
    assert all(t in (32, 64) for t in tiles) and all(min(p) > 0 for p in times)
    for i in range(len(tensors)):
        core, fac, r1 = ts.tucker_als_sketched(Tg[i], ranks[i], ms[i], sweeps, seed=seed + i)
        # the products are summed in another order (no split along m): FP32 rounding only
        assert abs(res[i] - float(r1[0])) <= 1e-4 * float(r1[0])
        for n in range(3):
            d = np.abs(proj(b.factors[i][n].cpu().numpy()) - proj(fac[n].cpu().numpy())).max()
            assert d < 1e-3
    b.close()


def test_batch_fp32_matches_oracle(ts):
    # 8 FP32 tensors of the batched workload's kind (uneven shapes and ranks, m = 8 R^2,
    # noise 1e-2) against the FP64 oracle run on each tensor's FP32 values with the same
    # seed: residuals and factor projectors at the FP32 tolerances of the single-tensor
    # tests.
    tensors, ranks, ms = batch_case(8, 6, np.float32, hi=96, rhi=9)
    sweeps, seed = 4, 21
    b = ts.TuckerBatch([torch.from_numpy(T).cuda() for T in tensors], ranks, ms, sweeps,
                       seed=seed)
    b.sweeps()
    res = b.residual().cpu().numpy()
    assert b.flags() == [0] * len(tensors)
    worst_r, worst_p = 0.0, 0.0
    for i, T in enumerate(tensors):
        T64 = T.astype(np.float64)
        c_o, f_o, _ = tucker.sketch_tucker_als(T64, ranks[i], ms[i], sweeps, seed=seed + i)
        r_o = tucker.residual(T64, c_o, f_o)
        worst_r = max(worst_r, abs(res[i] - r_o) / r_o)
        for n in range(3):
            worst_p = max(worst_p, np.abs(proj(b.factors[i][n].double().cpu().numpy()) -
                                          proj(f_o[n])).max())
    print({"residual": worst_r, "projector": worst_p})
    assert worst_r <= 1e-5 and worst_p <= 1e-4
    b.close()


def test_batch_sweeps_replay_as_a_cuda_graph(ts):
    tensors, ranks, ms = batch_case(6, 3, np.float32)
    Tg = [torch.from_numpy(T).cuda() for T in tensors]
    plain = ts.TuckerBatch(Tg, ranks, ms, 2, seed=5)
    plain.sweeps(0, 2)
    plain.sweeps(0, 2)
    graphed = ts.TuckerBatch(Tg, ranks, ms, 2, seed=5)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            graphed.sweeps(0, 2)
    torch.cuda.current_stream().wait_stream(s)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    r_plain = plain.residual().cpu().numpy()
    r_graph = graphed.residual().cpu().numpy()
    assert np.allclose(r_plain, r_graph, rtol=1e-4, atol=0)
    for i in range(len(tensors)):
        for n in range(3):
            a = proj(plain.factors[i][n].cpu().numpy())
            c = proj(graphed.factors[i][n].cpu().numpy())
            assert np.abs(a - c).max() < 1e-3
    plain.close()
    graphed.close()
