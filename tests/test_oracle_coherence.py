"""The tensor with large coherence (Sec. 7, Tensor 4) and the robustness it is used for.

Sec. 5 argues that leverage-score sampling started from random factors can miss the
few large entries of a highly coherent tensor, and that the range-finder
initialisation (Alg. 3) fixes this.  These tests check the generator against its
definition and that every sketch kind, started by Init-RRF, ends near HOOI on it.
"""

import numpy as np
import pytest

from oracle import tucker
from paper_2104_01101_gb300 import synth


def test_spiked_tensor_follows_its_definition():
    dims, ranks = (30, 20, 25), (4, 3, 5)
    X, pos, vals = synth.spiked_tucker(dims, ranks, 1e-3, seed=5, n_spikes=10)
    T, _, _ = synth.dense_tucker(dims, ranks, 1e-3, seed=5)
    D = X - T
    # exactly n entries differ, at distinct positions, by the returned values
    assert np.count_nonzero(D) == 10
    assert len({tuple(p) for p in pos}) == 10
    assert np.array_equal(D[tuple(pos.T)], vals)
    # each spike ~ N(||T|| / sqrt(n), 1): the norm ratio is about one
    ratio = np.linalg.norm(D) / np.linalg.norm(T)
    assert 0.6 < ratio < 1.5


def test_spiked_tensor_has_large_coherence():
    # The coherence of an orthonormal basis of the mode-1 unfolding's leading subspace
    # (Sec. 5 definition, with the square) is far above that of the plain Tucker tensor.
    def coherence(X, n, R):
        Xn = np.moveaxis(X, n, 0).reshape(X.shape[n], -1)
        U = np.linalg.svd(Xn, full_matrices=False)[0][:, :R]
        return X.shape[n] / R * np.max(np.sum(U * U, axis=1))
    dims, ranks = (40, 40, 40), (5, 5, 5)
    X, _, _ = synth.spiked_tucker(dims, ranks, 1e-3, seed=1)
    T, _, _ = synth.dense_tucker(dims, ranks, 1e-3, seed=1)
    for n in range(3):
        assert coherence(X, n, 5) > 2.0 * coherence(T, n, 5)


@pytest.mark.parametrize("kind", ["ts", "lev", "lev_det"])
def test_rrf_initialised_sketches_are_robust_on_tensor4(kind):
    # 40^3, rank 5, m = 16 R^2, 5 sweeps (Sec. 7's settings at the small size):
    # started by Init-RRF every sketch kind stays within 30 % of HOOI's residual.
    R = 5
    for gseed in range(2):
        X, _, _ = synth.spiked_tucker((40, 40, 40), (R, R, R), 1e-3, gseed)
        c, f = tucker.hooi(X, (R, R, R), 5)
        h = tucker.residual(X, c, f)
        for seed in range(2):
            c, f, _ = tucker.sketch_tucker_als(X, (R, R, R), 16 * R * R, 5, seed, kind=kind)
            assert tucker.residual(X, c, f) < 1.3 * h
