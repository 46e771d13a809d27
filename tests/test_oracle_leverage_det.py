"""Pins of the oracle's deterministic leverage selection ("Lev-fix", Sec. 3.2), CPU only."""

import itertools

import numpy as np
import pytest

from oracle import sketch, tucker
from paper_2104_01101_gb300 import synth


@pytest.mark.parametrize("sizes,m", [((7, 5), 9), ((4, 3, 5), 17), ((6, 6), 36), ((9,), 4)])
def test_selection_equals_brute_force(sizes, m):
    g = np.random.default_rng(1)
    scores = [g.random(s) for s in sizes]
    scores[0][1] = scores[0][2]          # a tie in one mode
    cand = []
    for lin, idx in enumerate(itertools.product(*[range(s) for s in sizes])):
        p = 1.0
        for k, i in enumerate(idx):
            p = p * scores[k][i]
        cand.append((-p, lin))
    want = sorted(lin for _, lin in sorted(cand)[:m])
    got = sketch.leverage_select_det(scores, m)
    assert list(got) == want


def test_ties_prefer_the_lower_linear_index():
    # all scores equal: the first m linear indices
    got = sketch.leverage_select_det([np.ones(4), np.full(5, 0.5)], 7)
    assert list(got) == list(range(7))


def test_selected_scores_dominate_the_rest():
    g = np.random.default_rng(2)
    scores = [g.random(8), g.random(6), g.random(5)]
    sel = sketch.leverage_select_det(scores, 31)
    full = np.einsum("a,b,c->abc", *scores).reshape(-1)
    rest = np.setdiff1d(np.arange(full.size), sel)
    assert full[sel].min() >= full[rest].max()


def test_all_rows_reduce_to_hooi():
    # m = prod of the other mode sizes keeps every row of P^(n): with the exact solve the
    # sketched ALS is HOOI from the same initial factors (Sec. 2.2, Alg. 1)
    dims, ranks = (7, 6, 5), (3, 2, 2)
    T, _, _ = synth.dense_tucker(dims, ranks, 0.3, seed=3)
    init = tucker.hosvd(T, ranks)
    m = max(dims[1] * dims[2], dims[0] * dims[2], dims[0] * dims[1])
    c_s, f_s, _ = tucker.sketch_tucker_als(T, ranks, m, 3, seed=0, kind="lev_det", solve="exact",
                                           init_factors=[None, init[1], init[2]])
    c_h, f_h = tucker.hooi(T, ranks, 3, init=init)
    for n in range(3):
        assert np.abs(f_s[n] @ f_s[n].T - f_h[n] @ f_h[n].T).max() < 1e-10
