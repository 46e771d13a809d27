"""Pins of the oracle's random objects (hash family, uniforms, Gaussians)."""

import os

import numpy as np
import pytest
from scipy import stats

from oracle import rng

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_outputs():
    # The generator advances its state by GAMMA and finalises; rand64 uses the same
    # finaliser, so it must reproduce the published sequence for state 0.
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        want = [int(l, 16) for l in f if l.strip() and not l.startswith("#")]
    got = [rng._mix64_int((i + 1) * rng.GAMMA) for i in range(len(want))]
    assert got == want
    # array version agrees with the scalar one
    z = np.array([(i + 1) * rng.GAMMA & rng.MASK64 for i in range(4)], dtype=np.uint64)
    assert [int(v) for v in rng._mix64(z)] == want


def test_rand64_definition():
    seed, tag = 12345, rng.make_tag(3, 7, 2, 1)
    key = rng._mix64_int(seed + rng.GAMMA * (tag + 1))
    for idx in (0, 1, 99, 2**40):
        want = rng._mix64_int(key + rng.GAMMA * (idx + 1))
        assert int(rng.rand64(seed, tag, idx)) == want


def test_poly_hash_matches_big_integer_evaluation():
    # Horner with a reduction per step == exact polynomial value mod p (Python ints).
    a, b = rng.hash_coefficients(7, rng.make_tag(1, 0, 0, 2))
    keys = np.array([0, 1, 2, 17, 399, 199999, 2**31 - 2], dtype=np.uint64)
    ga = rng.poly_mod_p(a, keys)
    gb = rng.poly_mod_p(b, keys)
    for j, x in enumerate(keys.tolist()):
        assert int(ga[j]) == sum(int(c) * x ** e for e, c in enumerate(a.tolist())) % rng.P31
        assert int(gb[j]) == sum(int(c) * x ** e for e, c in enumerate(b.tolist())) % rng.P31


def test_hash_table_uniform_buckets_and_balanced_signs():
    m, s = 97, 200000
    bins, signs = rng.hash_table(3, rng.PURPOSE_TS_HASH, 0, 0, 1, s, m)
    assert bins.min() >= 0 and bins.max() < m
    counts = np.bincount(bins, minlength=m)
    chi2 = ((counts - s / m) ** 2 / (s / m)).sum()
    assert stats.chi2.sf(chi2, m - 1) > 1e-4
    assert abs(signs.mean()) < 5.0 / np.sqrt(s)
    # pairwise: collisions among distinct keys happen at rate ~1/m
    i = np.arange(0, s - 1, 2)
    rate = np.mean(bins[i] == bins[i + 1])
    assert abs(rate - 1.0 / m) < 5 * np.sqrt((1 / m) / len(i))
    # pairwise sign products average ~0
    assert abs(np.mean(signs[i] * signs[i + 1])) < 5.0 / np.sqrt(len(i))


def test_tables_depend_on_every_tag_field():
    base = rng.hash_table(1, 1, 0, 0, 1, 1000, 50)[0]
    for args in [(2, 1, 0, 0, 1), (1, 2, 0, 0, 1), (1, 1, 1, 0, 1), (1, 1, 0, 1, 1), (1, 1, 0, 0, 2)]:
        other = rng.hash_table(args[0], args[1], args[2], args[3], args[4], 1000, 50)[0]
        assert np.mean(base == other) < 0.1


def test_pack_unpack_roundtrip():
    bins, signs = rng.hash_table(5, 1, 0, 1, 0, 5000, 4096)
    p = rng.pack_table(bins, signs)
    assert p.dtype == np.int32
    b2, s2 = rng.unpack_table(p)
    assert np.array_equal(b2, bins) and np.array_equal(s2, signs)


def test_uniform_and_gaussian_distributions():
    u = rng.uniform01(9, rng.make_tag(5, 0, 1, 2), np.arange(100000, dtype=np.uint64))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    g = rng.gaussian(9, rng.make_tag(4, 0, 1, 0), 100000)
    assert stats.kstest(g, "norm").pvalue > 1e-4
    assert abs(g.mean()) < 0.02 and abs(g.var() - 1.0) < 0.02


def test_gaussian_is_box_muller_of_the_counter_stream():
    seed, tag = 4, rng.make_tag(4, 1, 2, 0)
    g = rng.gaussian(seed, tag, 3)
    for e in range(3):
        r1 = int(rng.rand64(seed, tag, 2 * e))
        r2 = int(rng.rand64(seed, tag, 2 * e + 1))
        u1 = ((r1 >> 11) + 1) / 2.0 ** 53
        u2 = (r2 >> 11) / 2.0 ** 53
        import math
        assert g[e] == pytest.approx(math.sqrt(-2 * math.log(u1)) * math.cos(2 * math.pi * u2),
                                     rel=1e-14, abs=1e-14)
