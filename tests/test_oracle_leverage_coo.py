"""Pins of the oracle's leverage sampling on COO tensors (Sec. 3.2), CPU only.

The sampled right-hand side S T_(n)^T of a COO tensor is gathered from the nonzeros of
the sampled fibres; it must equal the same sampling applied to the densified tensor
(whose leverage sketch is pinned on its own), with repeated coordinates adding.
"""

import numpy as np
import pytest

from oracle import sketch, tucker
from paper_2104_01101_gb300 import synth


def _coo_with_duplicates(dims, nnz, seed):
    g = np.random.default_rng(seed)
    idx = np.stack([g.integers(0, s, nnz) for s in dims]).astype(np.int32)
    idx[:, nnz // 2:nnz // 2 + 5] = idx[:, :5]          # five repeated coordinates
    vals = g.standard_normal(nnz)
    return idx, vals


def _densify(idx, vals, dims):
    T = np.zeros(dims)
    for e in range(vals.shape[0]):
        T[tuple(int(idx[k, e]) for k in range(len(dims)))] += vals[e]
    return T


@pytest.mark.parametrize("dims,n", [((5, 6, 7), 0), ((5, 6, 7), 1), ((4, 3, 5, 2), 2)])
def test_fibre_rows_equal_brute_force(dims, n):
    idx, vals = _coo_with_duplicates(dims, 60, seed=3)
    g = np.random.default_rng(4)
    others = [k for k in range(len(dims)) if k != n]
    m = 9
    samples = np.stack([g.integers(0, dims[k], m) for k in others], axis=1)
    samples[3] = samples[1]                            # a repeated draw
    samples[5] = [int(idx[k, 0]) for k in others]      # a fibre holding a repeated entry
    w = g.random(m) + 0.5
    Y = sketch.fibre_rows_coo(idx, vals, dims, n, samples, w)
    for j in range(m):
        ref = np.zeros(dims[n])
        for e in range(vals.shape[0]):
            if all(int(idx[k, e]) == samples[j, c] for c, k in enumerate(others)):
                ref[int(idx[n, e])] += vals[e]
        assert np.allclose(Y[j], w[j] * ref, rtol=1e-15, atol=1e-15)


def test_empty_fibre_gives_a_zero_row():
    dims = (4, 5, 6)
    idx = np.array([[0, 1], [0, 2], [0, 3]], dtype=np.int32)
    Y = sketch.fibre_rows_coo(idx, np.array([2.0, 3.0]), dims, 0,
                              np.array([[4, 5], [0, 0], [2, 3]]), np.ones(3))
    assert np.array_equal(Y, np.array([[0, 0, 0, 0], [2.0, 0, 0, 0], [0, 3.0, 0, 0]]))


@pytest.mark.parametrize("det", [False, True])
def test_coo_sketch_equals_dense_sketch_of_the_densified_tensor(det):
    dims, n, m = (7, 6, 5), 1, 20
    idx, vals = _coo_with_duplicates(dims, 120, seed=5)
    T = _densify(idx, vals, dims)
    g = np.random.default_rng(6)
    factors = [synth.orthonormal(g, s, 3) for s in dims]
    if det:
        Zc, Yc, sc = sketch.leverage_sketch_coo_det(idx, vals, dims, n, factors, m)
        Zd, Yd, sd = sketch.leverage_sketch_dense_det(T, n, factors, m)
    else:
        Zc, Yc, sc, _ = sketch.leverage_sketch_coo(idx, vals, dims, n, factors, m, 11, 2)
        Zd, Yd, sd, _ = sketch.leverage_sketch_dense(T, n, factors, m, 11, 2)
    assert np.array_equal(sc, sd)
    assert np.array_equal(Zc, Zd)
    assert np.allclose(Yc, Yd, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("kind", ["lev", "lev_det"])
def test_coo_als_equals_dense_als(kind):
    # Sketched ALS on a sparse Tucker-structured COO tensor and on its densified copy.
    dims, ranks = (12, 10, 9), (3, 3, 2)
    idx, vals, _, _ = synth.coo_zipf_tucker(dims, 500, ranks, seed=7, val_dtype=np.float64)
    X = tucker.Coo(idx, vals, dims)
    T = _densify(idx, vals, dims)
    c1, f1, _ = tucker.sketch_tucker_als(X, ranks, 60, 3, seed=2, kind=kind)
    c2, f2, _ = tucker.sketch_tucker_als(T, ranks, 60, 3, seed=2, kind=kind)
    R1 = tucker.reconstruct(c1, f1)
    R2 = tucker.reconstruct(c2, f2)
    assert np.linalg.norm(R1 - R2) <= 1e-10 * np.linalg.norm(R2)
