"""Pins of the oracle's sketched-fit gradient (oracle/grad.py), CPU only.

The loss is quadratic in every single entry of the core and of each factor (Z is
linear in each factor, the model linear in A^(n) and in the core), so a central
difference is exact up to rounding: the gradient must match it to ~1e-9."""

import numpy as np
import pytest

from oracle import grad, rng
from oracle.tensor import reconstruct, ttm, unfold


def case(dims, ranks, n, m, seed=0):
    g = np.random.default_rng(seed)
    core = g.standard_normal(ranks)
    fac = [g.standard_normal((s, R)) for s, R in zip(dims, ranks)]
    tables = [rng.hash_table(3, 1, 0, n, k, dims[k], m) for k in range(len(dims)) if k != n]
    Y = g.standard_normal((m, dims[n]))
    return core, fac, tables, Y


@pytest.mark.parametrize("dims,ranks,n,m", [((5, 4, 3), (2, 3, 2), 1, 17),
                                            ((4, 3, 5, 3), (2, 2, 3, 2), 0, 23),
                                            ((6, 5), (3, 2), 1, 11),
                                            ((5, 4, 3), (2, 3, 2), 2, 7)])
def test_gradient_equals_central_differences(dims, ranks, n, m):
    core, fac, tables, Y = case(dims, ranks, n, m)
    _, gc, gA = grad.sketched_fit_grad(core, fac, Y, tables, n, m)
    h = 1e-3

    def fd(arr, idx):
        v = arr[idx]
        arr[idx] = v + h
        lp = grad.sketched_fit(core, fac, Y, tables, n, m)
        arr[idx] = v - h
        lm = grad.sketched_fit(core, fac, Y, tables, n, m)
        arr[idx] = v
        return (lp - lm) / (2 * h)

    for k in range(len(dims)):
        for idx in np.ndindex(*fac[k].shape):
            assert abs(fd(fac[k], idx) - gA[k][idx]) <= 1e-9 * max(1.0, abs(gA[k][idx]))
    for idx in np.ndindex(*ranks):
        assert abs(fd(core, idx) - gc[idx]) <= 1e-9 * max(1.0, abs(gc[idx]))


def test_identity_sketch_is_the_unsketched_fit():
    # Tables H_k(i) = i * stride, S = +1, m = prod s_k: S^(n) is the identity, so L is
    # 1/2 ||T~ - T||^2 and dL/dcore = (T~ - T) x_k A^(k)T for every k (a TTM chain).
    dims, ranks, n = (5, 4, 3), (2, 3, 2), 0
    g = np.random.default_rng(4)
    core = g.standard_normal(ranks)
    fac = [g.standard_normal((s, R)) for s, R in zip(dims, ranks)]
    T = g.standard_normal(dims)
    others = [k for k in range(3) if k != n]
    m = int(np.prod([dims[k] for k in others]))
    tables = []
    for j, k in enumerate(others):
        stride = int(np.prod([dims[l] for l in others[j + 1:]]))
        tables.append((np.arange(dims[k]) * stride, np.ones(dims[k])))
    Y = unfold(T, n).T
    loss, gc, gA = grad.sketched_fit_grad(core, fac, Y, tables, n, m)
    E = reconstruct(core, fac) - T
    assert abs(loss - 0.5 * np.sum(E * E)) <= 1e-12 * np.sum(E * E)
    want = E
    for k in range(3):
        want = ttm(want, fac[k].T, k)
    assert np.abs(gc - want).max() <= 1e-11 * np.abs(want).max()
    # dL/dA^(k) = E_(k) (C x_{j != k} A^(j))_(k)^T for every k, sketched modes included
    for k in range(3):
        B = core
        for j in range(3):
            if j != k:
                B = ttm(B, fac[j], j)
        wk = unfold(E, k) @ unfold(B, k).T
        assert np.abs(gA[k] - wk).max() <= 1e-11 * np.abs(wk).max()


def test_exact_model_has_zero_loss_and_gradient():
    dims, ranks, n, m = (6, 5, 4), (2, 2, 3), 1, 13
    core, fac, tables, _ = case(dims, ranks, n, m, seed=2)
    from oracle.sketch import input_sketch_dense
    Y = input_sketch_dense(reconstruct(core, fac), n, tables, m)
    loss, gc, gA = grad.sketched_fit_grad(core, fac, Y, tables, n, m)
    assert loss <= 1e-24
    assert np.abs(gc).max() <= 1e-12
    assert all(np.abs(a).max() <= 1e-12 for a in gA)
