"""Pins of the oracle's sketching operators (Sec. 3) against brute force and theory."""

import itertools

import numpy as np
import pytest
from scipy import stats

from oracle import rng, sketch
from oracle.tensor import kron_chain, unfold


def rand_tables(seed, dims, m):
    return [rng.hash_table(seed, rng.PURPOSE_TS_HASH, 0, 9, k, s, m) for k, s in enumerate(dims)]


def test_ts_hash_matches_one_based_formula_by_loops():
    # Paper's hash written 1-based: H(i) = (sum_n (H_n(i_n) - 1) mod m) + 1.
    dims, m = (3, 4, 5), 7
    tables = rand_tables(1, dims, m)
    H, S = sketch.ts_hash(tables, m)
    lin = 0
    for multi in itertools.product(*[range(s) for s in dims]):     # C order
        h1 = [tables[k][0][i] + 1 for k, i in enumerate(multi)]     # 1-based H_n
        want_h = (sum(h - 1 for h in h1) % m) + 1
        want_s = np.prod([tables[k][1][i] for k, i in enumerate(multi)])
        assert H[lin] + 1 == want_h and S[lin] == want_s
        lin += 1


def test_countsketch_matrix_structure():
    bins, signs = rng.hash_table(2, 1, 0, 0, 0, 50, 11)
    S = sketch.countsketch_matrix(bins, signs, 11)
    assert S.shape == (11, 50)
    assert np.all(np.count_nonzero(S, axis=0) == 1)
    assert np.array_equal(S[bins, np.arange(50)], signs)


@pytest.mark.parametrize("dims,ranks,m", [((6, 5), (3, 2), 13), ((4, 3, 5), (2, 3, 2), 30),
                                          ((5, 7), (4, 4), 16), ((3, 4, 2, 3), (2, 2, 2, 2), 11)])
def test_fft_identity_equals_countsketch_of_explicit_kronecker(dims, ranks, m):
    g = np.random.default_rng(0)
    factors = [g.standard_normal((s, R)) for s, R in zip(dims, ranks)]
    tables = rand_tables(3, dims, m)
    Z_fft = sketch.ts_apply_fft(factors, tables, m)
    # brute force: dense CountSketch matrix with the TensorSketch hash, times kron(P)
    H, S = sketch.ts_hash(tables, m)
    Sd = sketch.countsketch_matrix(H, S, m)
    Z_bf = Sd @ kron_chain(factors)
    assert np.allclose(Z_fft, Z_bf, rtol=1e-12, atol=1e-12 * np.abs(Z_bf).max())
    assert np.allclose(sketch.ts_apply_explicit(factors, tables, m), Z_bf, atol=1e-13)


def test_tensorsketch_norm_unbiased_over_seeds():
    # E ||S x||^2 = ||x||^2 for a CountSketch whose signs are (at least) pairwise independent;
    # the TensorSketch variance is at most (2 + 3^q) ||x||^4 / m for q sketched modes.
    dims, m = (6, 7), 25
    x = np.random.default_rng(1).standard_normal(np.prod(dims))
    vals = []
    for seed in range(3000):
        tables = [rng.hash_table(seed, 1, 0, 0, k, s, m) for k, s in enumerate(dims)]
        vals.append(np.sum((sketch.tensorsketch_sparse(tables, m) @ x) ** 2))
    vals = np.array(vals)
    x2 = np.dot(x, x)
    sigma = np.sqrt((2 + 3 ** len(dims)) * x2 ** 2 / m / len(vals))
    assert abs(vals.mean() - x2) < 5 * sigma


def test_input_sketch_dense_by_loops():
    dims, m = (4, 3, 5), 9
    T = np.random.default_rng(2).standard_normal(dims)
    for n in range(3):
        others = [k for k in range(3) if k != n]
        tables = [rng.hash_table(4, 1, 0, n, k, dims[k], m) for k in others]
        Y = np.zeros((m, dims[n]))
        for i in itertools.product(*[range(s) for s in dims]):
            b = sum(tables[j][0][i[k]] for j, k in enumerate(others)) % m
            sgn = np.prod([tables[j][1][i[k]] for j, k in enumerate(others)])
            Y[b, i[n]] += sgn * T[i]
        assert np.allclose(sketch.input_sketch_dense(T, n, tables, m), Y, atol=1e-13)


def test_input_sketch_coo_sums_duplicates_like_dense():
    dims, m = (5, 6, 4), 17
    g = np.random.default_rng(3)
    nnz = 300
    idx = np.stack([g.integers(0, s, nnz) for s in dims])
    vals = g.standard_normal(nnz)
    dense = np.zeros(dims)
    np.add.at(dense, tuple(idx), vals)
    for n in range(3):
        tables = sketch.ts_tables_for_mode(8, dims, n, m)
        assert np.allclose(sketch.input_sketch_coo(idx, vals, dims, n, tables, m),
                           sketch.input_sketch_dense(dense, n, tables, m), atol=1e-12)


def test_leverage_scores_definition_and_kronecker_lemma():
    g = np.random.default_rng(4)
    A1 = np.linalg.qr(g.standard_normal((9, 3)))[0]
    A2 = np.linalg.qr(g.standard_normal((7, 2)))[0]
    l1, l2 = sketch.leverage_scores(A1), sketch.leverage_scores(A2)
    assert l1.sum() == pytest.approx(3.0) and l2.sum() == pytest.approx(2.0)
    # definition with a non-orthonormal basis of the same column space: diag(QQ^T)
    B = A1 @ g.standard_normal((3, 3))
    Q = np.linalg.qr(B)[0]
    assert np.allclose(np.sum(Q * Q, axis=1), l1, atol=1e-13)
    # Kronecker lemma: scores of A1 (x) A2 are products of the factor scores
    P = np.kron(A1, A2)
    QP = np.linalg.qr(P)[0]
    assert np.allclose(np.sum(QP * QP, axis=1), np.kron(l1, l2), atol=1e-13)


def test_leverage_sampling_frequencies():
    ell = np.array([0.1, 0.5, 0.05, 0.9, 0.45])
    u = rng.uniform01(1, 77, np.arange(200000, dtype=np.uint64))
    idx, p = sketch.leverage_sample_mode(ell, u)
    counts = np.bincount(idx, minlength=5)
    expect = ell / ell.sum() * len(u)
    assert stats.chisquare(counts, expect).pvalue > 1e-4
    assert np.allclose(p, ell[idx] / ell.sum())
    # inverse-CDF rule: smallest i with cdf_i > u * total
    cdf = np.cumsum(ell)
    for j in range(50):
        i = idx[j]
        assert cdf[i] > u[j] * cdf[-1] and (i == 0 or cdf[i - 1] <= u[j] * cdf[-1])


def test_leverage_sketch_equals_explicit_sampling_matrix():
    g = np.random.default_rng(5)
    dims, ranks, m = (6, 5, 4), (2, 3, 2), 40
    T = g.standard_normal(dims)
    factors = [np.linalg.qr(g.standard_normal((s, R)))[0] for s, R in zip(dims, ranks)]
    n = 1
    Z, Y, samples, w = sketch.leverage_sketch_dense(T, n, factors, m, seed=3, sweep=0)
    others = [0, 2]
    # explicit S = D Omega over the rows of P^(n) (C order over modes 0, 2)
    S = np.zeros((m, dims[0] * dims[2]))
    for j in range(m):
        S[j, samples[j, 0] * dims[2] + samples[j, 1]] = w[j]
    P = kron_chain([factors[k] for k in others])
    assert np.allclose(Z, S @ P, atol=1e-13)
    assert np.allclose(Y, S @ unfold(T, n).T, atol=1e-13)
    # weights follow the importance-sampling definition with p = prod_k l/R_k
    p = np.ones(m)
    for j, k in enumerate(others):
        p *= sketch.leverage_scores(factors[k])[samples[:, j]] / ranks[k]
    assert np.allclose(w, 1.0 / np.sqrt(m * p))


def test_leverage_sketch_is_unbiased_embedding():
    # E[S^T S] = I  =>  E[Z^T Z] = P^T P = I for orthonormal factors.
    g = np.random.default_rng(6)
    dims, ranks, m = (8, 8, 8), (2, 2, 2), 30
    T = g.standard_normal(dims)
    factors = [np.linalg.qr(g.standard_normal((s, R)))[0] for s, R in zip(dims, ranks)]
    acc = np.zeros((4, 4))
    trials = 1500
    for seed in range(trials):
        Z, _, _, _ = sketch.leverage_sketch_dense(T, 0, factors, m, seed=seed, sweep=0)
        acc += Z.T @ Z
    assert np.allclose(acc / trials, np.eye(4), atol=0.08)
