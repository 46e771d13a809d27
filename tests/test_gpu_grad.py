"""Gradient of the sketched fit (ts_fit_grad / SketchedFit) on the GPU against the FP64
oracle's explicit-matrix gradient and against central finite differences."""

import numpy as np
import pytest
import torch

from oracle import grad, rng, sketch
from paper_2104_01101_gb300 import synth

from bounds import U32, fit_grad_abs, fit_grad_depth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ts():
    from paper_2104_01101_gb300 import build, tsketch
    build.build_library()
    tsketch.lib()
    return tsketch


def tables_for(dims, n, m, seed=5):
    host = {k: rng.hash_table(seed, 1, 0, n, k, dims[k], m) for k in range(len(dims)) if k != n}
    dev = [torch.from_numpy(rng.pack_table(*host[k])).cuda() if k in host else None
           for k in range(len(dims))]
    return [host[k] for k in sorted(host)], dev


@pytest.mark.parametrize("dims,ranks,n,m", [((12, 10, 9), (3, 4, 2), 0, 60),
                                            ((12, 10, 9), (3, 4, 2), 1, 97),
                                            ((8, 7, 6, 5), (2, 3, 2, 2), 2, 64),
                                            ((30, 30, 30), (25, 25, 25), 0, 3000)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_fit_grad_matches_oracle(ts, dims, ranks, n, m, dtype):
    g = np.random.default_rng(3)
    core = g.standard_normal(ranks)
    fac = [np.linalg.qr(g.standard_normal((s, R)))[0] for s, R in zip(dims, ranks)]
    T = g.standard_normal(dims)
    host_tabs, dev_tabs = tables_for(dims, n, m)
    Y = sketch.input_sketch_dense(T, n, host_tabs, m)
    if dtype == torch.float32:  # the oracle sees the FP32-rounded inputs
        core, fac, Y = (core.astype(np.float32).astype(np.float64),
                        [f.astype(np.float32).astype(np.float64) for f in fac],
                        Y.astype(np.float32).astype(np.float64))
    L_o, gc_o, gA_o = grad.sketched_fit_grad(core, fac, Y, host_tabs, n, m)
    cast = lambda a: torch.from_numpy(a).to(dtype).cuda()
    L, gc, gA = ts.fit_grad(cast(core), [cast(f) for f in fac], cast(Y), dev_tabs, n, m)
    if dtype == torch.float64:
        tol = 1e-10
        assert abs(float(L) - L_o) <= tol * L_o
        assert np.linalg.norm(gc.double().cpu().numpy() - gc_o) <= tol * np.linalg.norm(gc_o)
        for k in range(len(dims)):
            d = np.linalg.norm(gA[k].double().cpu().numpy() - gA_o[k])
            assert d <= tol * np.linalg.norm(gA_o[k])
        return
    # FP32: the gradient sums terms of both signs (Z^T R, and R = Z M - Y itself), so its
    # error is relative to the same chain run on absolute values, not to the gradient:
    # first order, ||error|| <= depth u ||gradient of |.| chain|| with depth the roundings
    # along the longest chain (m terms in Z^T R dominate at m = 3000)
    assert abs(float(L) - L_o) <= 1e-5 * L_o
    gc_b, gA_b = fit_grad_abs(core, fac, Y, host_tabs, n, m)
    c = fit_grad_depth(dims, ranks, n, m) * U32
    assert np.linalg.norm(gc.double().cpu().numpy() - gc_o) <= c * np.linalg.norm(gc_b)
    for k in range(len(dims)):
        assert np.linalg.norm(gA[k].double().cpu().numpy() - gA_o[k]) <= c * np.linalg.norm(gA_b[k])


def test_fit_grad_central_differences_on_a_30_cube_slice(ts):
    # The collinear-CP workload's tensor, a 30^3 slice, Tucker (25, 25, 25), m = 3000:
    # central differences with h = 1e-3 in FP64 through the GPU loss (exact up to
    # rounding: the loss is quadratic in every single entry).
    T, _ = synth.cp_collinear((30, 30, 30), 20, 0.9, 1e-2, seed=4)
    dims, ranks, n, m = T.shape, (25, 25, 25), 1, 3000
    from oracle.tucker import hosvd
    from oracle.tensor import ttm
    fac = hosvd(T, ranks)
    core = T
    for k in range(3):
        core = ttm(core, fac[k].T, k)
    g = np.random.default_rng(8)
    core = core + 0.1 * g.standard_normal(ranks)   # away from the optimum
    host_tabs, dev_tabs = tables_for(dims, n, m, seed=9)
    Y = torch.from_numpy(sketch.input_sketch_dense(T, n, host_tabs, m)).cuda()
    core_t = torch.from_numpy(core).cuda()
    fac_t = [torch.from_numpy(f).cuda() for f in fac]
    _, gc, gA = ts.fit_grad(core_t, fac_t, Y, dev_tabs, n, m)
    h = 1e-3

    def loss():
        return float(ts.fit_grad(core_t, fac_t, Y, dev_tabs, n, m)[0])

    picks = [(None, (3, 4, 5)), (None, (24, 0, 11)), (0, (7, 3)), (1, (29, 24)), (2, (0, 0)),
             (2, (15, 12))]
    for k, idx in picks:
        arr = core_t if k is None else fac_t[k]
        want = (gc if k is None else gA[k])[idx].item()
        v = arr[idx].item()
        arr[idx] = v + h
        lp = loss()
        arr[idx] = v - h
        lm = loss()
        arr[idx] = v
        fd = (lp - lm) / (2 * h)
        assert abs(fd - want) <= 1e-7 * max(1.0, abs(want))


def test_autograd_function_backward(ts):
    dims, ranks, n, m = (10, 9, 8), (3, 2, 3), 2, 50
    g = np.random.default_rng(1)
    host_tabs, dev_tabs = tables_for(dims, n, m)
    Y = torch.from_numpy(g.standard_normal((m, dims[n]))).cuda()
    core = torch.from_numpy(g.standard_normal(ranks)).cuda().requires_grad_()
    fac = [torch.from_numpy(g.standard_normal((s, R))).cuda().requires_grad_()
           for s, R in zip(dims, ranks)]
    L = ts.sketched_fit(core, fac, Y, dev_tabs, n, m)
    (3.0 * L).backward()
    L_o, gc_o, gA_o = grad.sketched_fit_grad(core.detach().cpu().numpy(),
                                             [f.detach().cpu().numpy() for f in fac],
                                             Y.cpu().numpy(), host_tabs, n, m)
    assert abs(float(L.detach()) - L_o) <= 1e-10 * L_o
    assert np.abs(core.grad.cpu().numpy() - 3.0 * gc_o).max() <= 1e-9 * np.abs(gc_o).max()
    for k in range(3):
        assert np.abs(fac[k].grad.cpu().numpy() - 3.0 * gA_o[k]).max() <= 1e-9 * np.abs(gA_o[k]).max()


def test_loss_only_call_skips_the_gradient(ts):
    # Without requires_grad the autograd function asks the library for the loss alone
    # (null gradient outputs: no backward products, no adjoint FFT chain); the loss is the
    # same as the one computed with the gradients.
    dims, ranks, n, m = (10, 9, 8), (3, 2, 3), 1, 50
    g = np.random.default_rng(2)
    host_tabs, dev_tabs = tables_for(dims, n, m)
    Y = torch.from_numpy(g.standard_normal((m, dims[n]))).cuda()
    core = torch.from_numpy(g.standard_normal(ranks)).cuda()
    fac = [torch.from_numpy(g.standard_normal((s, R))).cuda() for s, R in zip(dims, ranks)]
    l0 = ts.kernel_launches()
    L = ts.sketched_fit(core, fac, Y, dev_tabs, n, m)
    loss_only = ts.kernel_launches() - l0
    l0 = ts.kernel_launches()
    L2, gc, _ = ts.fit_grad(core, fac, Y, dev_tabs, n, m)
    with_grad = ts.kernel_launches() - l0
    assert loss_only < with_grad
    assert abs(float(L) - float(L2)) <= 1e-12 * abs(float(L2))
    L_o = grad.sketched_fit(core.cpu().numpy(), [f.cpu().numpy() for f in fac], Y.cpu().numpy(),
                            host_tabs, n, m)
    assert abs(float(L) - L_o) <= 1e-10 * L_o

