"""Parity of each hot-path row (CUDA via the C ABI) against the FP64 oracle."""

import numpy as np
import pytest
import torch

import oracle
from oracle import rng, sketch, solve, tucker
from paper_2104_01101_gb300 import synth

from bounds import (U32, U64, input_sketch_coo_terms, input_sketch_terms, summation_bound,
                    ts_fft_column_bound, unit_tables)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ts():
    from paper_2104_01101_gb300 import build, tsketch
    build.build_library()
    tsketch.lib()
    return tsketch


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def packed_tables(seed, dims, n, m, purpose=1, sweep=0):
    out = {}
    for k in range(len(dims)):
        if k != n:
            b, s = rng.hash_table(seed, purpose, sweep, n, k, dims[k], m)
            out[k] = (b, s, dev(rng.pack_table(b, s)))
    return out


# ---------------------------------------------------------------- a1 hash tables

@pytest.mark.parametrize("purpose,sweep,n,k,size,nbins", [
    (1, 0, 0, 1, 40, 400), (1, 0, 2, 1, 400, 2000), (2, 0, 1, 0, 4000, 115),
    (1, 7, 3, 2, 200000, 4096), (1, 0, 0, 0, 1, 1), (2, 3, 255, 255, 3001, 97)])
def test_hash_tables_bit_exact(ts, purpose, sweep, n, k, size, nbins):
    seed = 0xDEADBEEF12345
    got = ts.hash_table(seed, purpose, sweep, n, k, size, nbins).cpu().numpy()
    b, s = rng.hash_table(seed, purpose, sweep, n, k, size, nbins)
    assert np.array_equal(got, rng.pack_table(b, s))


# ---------------------------------------------------------------- a2 + a3 TensorSketch of a chain

@pytest.mark.parametrize("dims,ranks,m", [
    ((40, 40), (5, 5), 400),            # small dense workload shapes
    ((400, 400), (10, 10), 2000),       # 400^3 workload shapes
    ((33, 29, 17), (3, 4, 2), 210),     # three factors, m = 2*3*5*7
    ((50,), (7,), 128),                 # single factor (order-2 tensors)
    ((21, 19), (4, 3), 2 * 97),         # large prime factor in m
    ((300, 300), (25, 25), 3000),       # 300^3 rank-25 shapes
])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_tensorsketch_apply_matches_explicit_kronecker(ts, dims, ranks, m, dtype):
    g = np.random.default_rng(1)
    factors = [np.linalg.qr(g.standard_normal((s, R)))[0] for s, R in zip(dims, ranks)]
    tabs = [rng.hash_table(5, 1, 0, 9, j, s, m) for j, s in enumerate(dims)]
    if np.prod(dims) * np.prod(ranks) <= 3e7:
        want = sketch.ts_apply_explicit(factors, tabs, m)
    else:
        want = sketch.ts_apply_fft(factors, tabs, m)
    Z = ts.tensorsketch_apply([dev(f, dtype) for f in factors],
                              [dev(rng.pack_table(*t)) for t in tabs], m).cpu().numpy()
    tol = 1e-12 if dtype == torch.float64 else 1e-5
    assert np.linalg.norm(Z - want) <= tol * np.linalg.norm(want)
    # element-wise: every entry within the FFT-convolution bound of its column
    u = U64 if dtype == torch.float64 else U32
    assert np.all(np.abs(Z - want) <= ts_fft_column_bound(factors, tabs, m, u))


# ---------------------------------------------------------------- a4 input sketch

@pytest.mark.parametrize("dims,m", [((40, 40, 40), 400), ((13, 7, 11), 50), ((9, 8, 7, 6), 300),
                                    ((64, 3), 17), ((50, 100, 172), 300)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_input_sketch_dense(ts, dims, m, dtype):
    T = np.random.default_rng(2).standard_normal(dims)
    Tg = dev(T, dtype)
    for n in range(len(dims)):
        tabs = packed_tables(7, dims, n, m)
        Y = ts.tensorsketch_input(Tg, n, [tabs[k][2] if k in tabs else None
                                          for k in range(len(dims))], m).cpu().numpy()
        Tx = T.astype(np.float64) if dtype == torch.float64 else \
            T.astype(np.float32).astype(np.float64)
        host = [tabs[k][:2] for k in sorted(tabs)]
        want = sketch.input_sketch_dense(Tx, n, host, m)
        tol = 1e-12 if dtype == torch.float64 else 1e-5
        assert np.linalg.norm(Y - want) <= tol * np.linalg.norm(want)
        # element-wise: any-order summation of each bin's terms, plus (FP32, first mode of
        # an order-3 tensor) the fixed-point quantisation of at most max|T slice| 2^-19 a term
        absY, cnt = input_sketch_terms(Tx, n, host, m)
        bound = summation_bound(absY, cnt, U64 if dtype == torch.float64 else U32)
        if dtype == torch.float32 and n == 0 and len(dims) == 3:
            bound = bound + cnt * np.abs(Tx).reshape(dims[0], -1).max(axis=1)[None, :] * 2.0 ** -19
        assert np.all(np.abs(Y - want) <= bound + 1e-300)


@pytest.mark.parametrize("case", ["late_spikes", "scaled_slices", "one_bucket_tables"])
def test_input_sketch_dense_fixed_point_edges(ts, case):
    # The FP32 order-3 kernel keeps each slice's mode-1 buckets in 32-bit fixed point
    # scaled by the largest value of the slice's first tile; larger values take an FP32
    # path, and tables that send too many entries to one bucket disable fixed point.
    dims, m = (50, 100, 172), 300
    g = np.random.default_rng(11)
    T = g.standard_normal(dims).astype(np.float32)
    if case == "late_spikes":
        T[::7, -1, -4:] = 3e4          # in the last tile of those slices
    if case == "scaled_slices":
        T *= (10.0 ** g.integers(-6, 4, size=dims[0]))[:, None, None].astype(np.float32)
    tabs = packed_tables(13, dims, 0, m)
    if case == "one_bucket_tables":
        for k in (1, 2):
            b, sg = tabs[k][:2]
            b = np.zeros_like(b)
            tabs[k] = (b, sg, dev(rng.pack_table(b, sg)))
    Y = ts.tensorsketch_input(dev(T), 0, [None, tabs[1][2], tabs[2][2]], m).cpu().numpy()
    want = sketch.input_sketch_dense(T.astype(np.float64), 0, [tabs[1][:2], tabs[2][:2]], m)
    # FP32 summation error is relative to the sum of |terms| of each bucket: with one
    # bucket per slice (17200 cancelling terms) that, not the sum, is the scale
    ref = want
    if case == "one_bucket_tables":
        ref = sketch.input_sketch_dense(np.abs(T).astype(np.float64), 0,
                                        [(tabs[k][0], np.ones_like(tabs[k][1])) for k in (1, 2)], m)
    for i in range(dims[0]):
        assert np.linalg.norm(Y[:, i] - want[:, i]) <= 1e-5 * np.linalg.norm(ref[:, i])
    absY, cnt = input_sketch_terms(T.astype(np.float64), 0, [tabs[1][:2], tabs[2][:2]], m)
    quant = cnt * np.abs(T).reshape(dims[0], -1).max(axis=1)[None, :].astype(np.float64) * 2.0 ** -19
    assert np.all(np.abs(Y - want) <= summation_bound(absY, cnt, U32) + quant)


def test_input_sketch_dense_full_size_sampled_columns(ts):
    # The 400^3 FP32 workload: compare a few whole columns Y_n[:, i] with the oracle
    # applied to the slab T(i along mode n), plus the squared-norm invariant.
    dims, m = (400, 400, 400), 2000
    T, _, _ = synth.dense_tucker(dims, (10, 10, 10), 1e-2, seed=5, core_decay=0.9,
                                 dtype=np.float32)
    Tg = dev(T)
    for n in range(3):
        tabs = packed_tables(9, dims, n, m)
        Y = ts.tensorsketch_input(Tg, n, [tabs[k][2] if k in tabs else None for k in range(3)], m)
        Y = Y.cpu().numpy().astype(np.float64)
        host = [tabs[k][:2] for k in sorted(tabs)]
        S = sketch.tensorsketch_sparse(host, m)
        Su = sketch.tensorsketch_sparse(unit_tables(host), m)
        for i in (0, 17, 399):
            slab = np.take(T, i, axis=n).astype(np.float64).reshape(-1)
            want = S @ slab
            assert np.linalg.norm(Y[:, i] - want) <= 1e-5 * np.linalg.norm(want)
            cnt = Su @ np.ones_like(slab)
            bound = cnt * U32 * (Su @ np.abs(slab))
            if n == 0:  # fixed-point buckets of the first mode
                bound = bound + cnt * np.abs(slab).max() * 2.0 ** -19
            assert np.all(np.abs(Y[:, i] - want) <= bound)


def test_input_sketch_coo_full_size_sampled_columns(ts):
    # The full sparse 4-way workload: dims 2e5 per mode, 1e8 Zipf(1.1) coordinates with
    # duplicates, m = 4096.  Whole columns Y_n[:, i] are recomputed by the oracle from the
    # nonzeros with i_n = i (the Zipf head index 0 alone has ~1e7 of them).
    dims, nnz, m = (200_000,) * 4, 100_000_000, 4096
    idx, vals = synth.coo_zipf_tucker_torch(dims, nnz, (8, 8, 8, 8), seed=3, device="cuda")
    X = ts.Coo(idx, vals, dims)
    for n in (0, 3):
        tabs = packed_tables(21, dims, n, m)
        Y = ts.tensorsketch_input(X, n, [tabs[k][2] if k in tabs else None for k in range(4)], m)
        host_tabs = [tabs[k][:2] for k in sorted(tabs)]
        for i in (0, 1, 777, 150_000):
            sel = idx[n] == i
            sub_idx = idx[:, sel].cpu().numpy().astype(np.int64)
            sub_vals = vals[sel].cpu().numpy()
            sub_idx[n] = 0                       # one column: mode n of extent 1
            d1 = list(dims)
            d1[n] = 1
            want = sketch.input_sketch_coo(sub_idx, sub_vals, d1, n, host_tabs, m)[:, 0]
            scale = sketch.input_sketch_coo(sub_idx, np.abs(sub_vals), d1, n,
                                            [(b, np.ones_like(sg)) for b, sg in host_tabs], m)[:, 0]
            got = Y[:, i].double().cpu().numpy()
            assert np.linalg.norm(got - want) <= 1e-5 * max(np.linalg.norm(scale), 1e-30)
            cnt = sketch.input_sketch_coo(sub_idx, np.ones(sub_vals.shape[0]), d1, n,
                                          [(b, np.ones_like(sg)) for b, sg in host_tabs], m)[:, 0]
            assert np.all(np.abs(got - want) <= cnt * U32 * scale)
        del Y


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_input_sketch_coo_with_duplicates_and_empty(ts, dtype):
    dims, m = (2000, 1500, 1000, 700), 512
    idx, vals, _, _ = synth.coo_zipf_tucker(dims, 200000, (3, 3, 3, 3), seed=4,
                                            val_dtype=np.float64)
    X = ts.Coo(dev(idx), dev(vals, dtype), dims)
    for n in range(4):
        tabs = packed_tables(3, dims, n, m)
        Y = ts.tensorsketch_input(X, n, [tabs[k][2] if k in tabs else None for k in range(4)], m)
        want = sketch.input_sketch_coo(idx, vals if dtype == torch.float64 else
                                       vals.astype(np.float32).astype(np.float64),
                                       dims, n, [tabs[k][:2] for k in sorted(tabs)], m)
        tol = 1e-12 if dtype == torch.float64 else 1e-5
        assert np.linalg.norm(Y.cpu().numpy() - want) <= tol * np.linalg.norm(want)
        vx = vals if dtype == torch.float64 else vals.astype(np.float32).astype(np.float64)
        absY, cnt = input_sketch_coo_terms(idx, vx, dims, n, [tabs[k][:2] for k in sorted(tabs)], m)
        u = U64 if dtype == torch.float64 else U32
        assert np.all(np.abs(Y.cpu().numpy() - want) <= summation_bound(absY, cnt, u) + 1e-300)
    empty = ts.Coo(torch.zeros((4, 0), dtype=torch.int32, device="cuda"),
                   torch.zeros(0, dtype=dtype, device="cuda"), dims)
    tabs = packed_tables(3, dims, 0, m)
    Y = ts.tensorsketch_input(empty, 0, [tabs[k][2] if k in tabs else None for k in range(4)], m)
    assert float(Y.abs().max()) == 0.0


# ---------------------------------------------------------------- a6 Init-RRF

@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-10), (torch.float32, 1e-5)])
def test_range_finder_matches_oracle(ts, dtype, tol):
    dims, ranks = (40, 36, 30), (5, 4, 6)
    T, _, _ = synth.dense_tucker(dims, ranks, 1e-3, seed=6)
    Tx = T if dtype == torch.float64 else T.astype(np.float32).astype(np.float64)
    for n in (1, 2):
        k1, k2 = tucker.rrf_sizes(dims, n, ranks[n], 400)
        A = ts.range_finder_init(dev(T, dtype), n, ranks[n], k1, k2, seed=21).cpu().numpy()
        want = tucker.init_rrf(Tx, n, ranks[n], k1, k2, seed=21)
        assert np.abs(A - want).max() <= tol * 10
        assert np.abs(A @ A.T - want @ want.T).max() <= tol


# ---------------------------------------------------------------- a7 + a8 sketched solve

def _solve_problem(seed, m, r, s, R, noise):
    g = np.random.default_rng(seed)
    Z = g.standard_normal((m, r)) / np.sqrt(m)
    X0 = g.standard_normal((r, R)) @ g.standard_normal((R, s))
    return Z, Z @ X0 + noise * g.standard_normal((m, s))


# The single-block Gauss-Jordan cuts its rank-16 update into 8-row items, or 10-row
# items when 8 would give some update warp a second item: r = 100, 105, 110, 120 take
# 10-row items (straddling the 16-row panels; r = 105 overhangs the last one), r = 125
# falls back to 8-row items in several rounds, r = 13 and 25 fit 8-row items.
@pytest.mark.parametrize("m,r,s,R", [(400, 25, 40, 5), (2000, 100, 400, 10), (97, 13, 31, 3),
                                     (3000, 125, 300, 12), (1500, 120, 200, 3),
                                     (1500, 105, 300, 6), (1500, 110, 300, 6)])
@pytest.mark.parametrize("dtype,fp64", [(torch.float64, False), (torch.float32, False),
                                        (torch.float32, True)],
                         ids=["f64", "f32", "f32-fp64-qr-svd"])
def test_rsvd_lrls_matches_oracle(ts, m, r, s, R, dtype, fp64):
    # fp64: the precision form (FP32 data; the QR of C and the eigen-decomposition of the
    # truncation's Gram in FP64)
    Z, Y = _solve_problem(3, m, r, s, R, 0.05)
    if dtype == torch.float32:
        Z = Z.astype(np.float32).astype(np.float64)
        Y = Y.astype(np.float32).astype(np.float64)
    k = solve.rsvd_oversampled_rank(R, 5, r, s)
    Om = rng.gaussian(77, rng.make_tag(4, 2, 1, 0), s * k).reshape(s, k)
    Cw, Aw = solve.rsvd_lrls(Z, Y, R, Om)
    Cg, Ag = ts.lrls_solve(dev(Z, dtype), dev(Y, dtype), R, ts.SOLVE_RSVD, seed=77, sweep=2, n=1,
                           solve_fp64=fp64)
    Bw, Bg = Cw @ Aw.T, Cg.cpu().numpy() @ Ag.cpu().numpy().T
    tol = 1e-11 if dtype == torch.float64 else 1e-5
    assert np.linalg.norm(Bg - Bw) <= tol * np.linalg.norm(Bw)
    assert np.abs(Ag.cpu().numpy() - Aw).max() <= (1e-9 if dtype == torch.float64 else 1e-4)


@pytest.mark.parametrize("m,r,s,R,k", [(600, 225, 20000, 3, None), (700, 64, 70000, 8, None),
                                       (512, 300, 17000, 20, 28)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_rsvd_lrls_wide_s_matches_oracle(ts, m, r, s, R, k, dtype):
    # s >= 16384 (a mode size of the sparse workloads): Y Omega and D = (Z E)^T Y take the
    # one-pass products over Y (split over s; k sums per column), the factor signs the
    # multi-block finalize; r s > 2^22 keeps the multi-kernel solve.  k = 28 takes the
    # 32-wide register form of the D product.
    Z, Y = _solve_problem(4, m, r, s, R, 0.05)
    if dtype == torch.float32:
        Z = Z.astype(np.float32).astype(np.float64)
        Y = Y.astype(np.float32).astype(np.float64)
    p = 5 if k is None else k - R
    kk = solve.rsvd_oversampled_rank(R, p, r, s)
    Om = rng.gaussian(91, rng.make_tag(4, 1, 0, 0), s * kk).reshape(s, kk)
    Cw, Aw = solve.rsvd_lrls(Z, Y, R, Om)
    Cg, Ag = ts.lrls_solve(dev(Z, dtype), dev(Y, dtype), R, ts.SOLVE_RSVD, seed=91, sweep=1, n=0,
                           oversample=p)
    Bw, Bg = Cw @ Aw.T, Cg.cpu().numpy() @ Ag.cpu().numpy().T
    tol = 1e-11 if dtype == torch.float64 else 2e-5
    assert np.linalg.norm(Bg - Bw) <= tol * np.linalg.norm(Bw)


@pytest.mark.parametrize("dtype,m,r,s,R", [(torch.float32, 2048, 256, 3000, 8),
                                           (torch.float32, 3000, 625, 300, 25),
                                           (torch.float64, 2048, 256, 3000, 8),
                                           (torch.float64, 3000, 512, 2000, 8)])
def test_rsvd_lrls_large_r_matches_oracle(ts, dtype, m, r, s, R):
    # r too large for the on-chip factorization: G^{-1} by Newton-Schulz products, whose
    # early stop must leave the inverse at the rounding floor (FP64: 1e-11 as the other
    # FP64 solves; r = 512 is the largest FP64 core whose QR fits one block)
    Z, Y = _solve_problem(6, m, r, s, R, 0.05)
    if dtype == torch.float32:
        Z = Z.astype(np.float32).astype(np.float64)
        Y = Y.astype(np.float32).astype(np.float64)
    k = solve.rsvd_oversampled_rank(R, 5, r, s)
    Om = rng.gaussian(5, rng.make_tag(4, 0, 2, 0), s * k).reshape(s, k)
    Cw, Aw = solve.rsvd_lrls(Z, Y, R, Om)
    Cg, Ag = ts.lrls_solve(dev(Z, dtype), dev(Y, dtype), R, ts.SOLVE_RSVD, seed=5, sweep=0, n=2)
    Bw, Bg = Cw @ Aw.T, Cg.cpu().numpy() @ Ag.cpu().numpy().T
    tol = 1e-5 if dtype == torch.float32 else 1e-11
    assert np.linalg.norm(Bg - Bw) <= tol * np.linalg.norm(Bw)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_exact_lrls_matches_oracle(ts, dtype):
    Z, Y = _solve_problem(4, 400, 25, 40, 5, 0.1)
    if dtype == torch.float32:
        Z = Z.astype(np.float32).astype(np.float64)
        Y = Y.astype(np.float32).astype(np.float64)
    Cw, Aw = solve.lrls_exact(Z, Y, 5)
    Cg, Ag = ts.lrls_solve(dev(Z, dtype), dev(Y, dtype), 5, ts.SOLVE_EXACT)
    Bw, Bg = Cw @ Aw.T, Cg.cpu().numpy() @ Ag.cpu().numpy().T
    tol = 1e-11 if dtype == torch.float64 else 1e-5
    assert np.linalg.norm(Bg - Bw) <= tol * np.linalg.norm(Bw)


def test_rsvd_exact_rank_input_equals_exact_solve(ts):
    # noiseless rank-R right-hand side: RSVD-LRLS is exact (degenerate case of Alg. 5)
    Z, Y = _solve_problem(5, 300, 20, 60, 4, 0.0)
    C1, A1 = ts.lrls_solve(dev(Z), dev(Y), 4, ts.SOLVE_RSVD, seed=1)
    C2, A2 = ts.lrls_solve(dev(Z), dev(Y), 4, ts.SOLVE_EXACT)
    B1 = (C1 @ A1.t()).cpu().numpy()
    B2 = (C2 @ A2.t()).cpu().numpy()
    assert np.linalg.norm(B1 - B2) <= 1e-10 * np.linalg.norm(B2)


# ---------------------------------------------------------------- a5 leverage sampling

@pytest.mark.parametrize("dims,mode,m,ties", [((40, 40, 40), 0, 400, False),
                                              ((40, 40, 40), 2, 2000, False),
                                              ((12, 10, 9, 8), 1, 150, False),
                                              ((16, 12, 10), 0, 50, True)])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_leverage_det_sketch_matches_oracle(ts, dims, mode, m, ties, dtype):
    # deterministic selection: the same multi-indices as the oracle (bit-exact), rows
    # beyond prod dims zero (m = 2000 > 1600), ties (equal row norms) to the lower index
    g = np.random.default_rng(4)
    T = g.standard_normal(dims)
    R = 3
    fac = [np.linalg.qr(g.standard_normal((s, R)))[0] for s in dims]
    if ties:
        for k in range(len(dims)):
            fac[k] = np.zeros((dims[k], R))
            fac[k][np.arange(dims[k]), np.arange(dims[k]) % R] = 1.0  # equal row norms
    if dtype == torch.float32:
        T = T.astype(np.float32).astype(np.float64)
        fac = [f.astype(np.float32).astype(np.float64) for f in fac]
    Zw, Yw, sw = sketch.leverage_sketch_dense_det(T, mode, fac, m)
    Zg, Yg, sg = ts.leverage_sketch_det(dev(T, dtype), mode, [dev(f, dtype) for f in fac], m)
    nsel = sw.shape[0]
    assert np.array_equal(sg.cpu().numpy()[:nsel], sw.astype(np.int32))
    tol = 1e-14 if dtype == torch.float64 else 1e-6
    Zg, Yg = Zg.double().cpu().numpy(), Yg.double().cpu().numpy()
    assert np.abs(Zg[:nsel] - Zw).max() <= tol * max(1.0, np.abs(Zw).max())
    assert np.abs(Yg[:nsel] - Yw).max() <= tol * max(1.0, np.abs(Yw).max())
    assert not np.any(Zg[nsel:]) and not np.any(Yg[nsel:])

@pytest.mark.parametrize("dims,ranks,m", [((40, 40, 40), (5, 5, 5), 400), ((30, 20, 25, 10), (3, 2, 4, 2), 300)])
def test_leverage_sketch_samples_bit_exact(ts, dims, ranks, m):
    T, _, A = synth.dense_tucker(dims, ranks, 0.01, seed=8)
    Tg = dev(T)
    Ag = [dev(a) for a in A]
    for n in range(len(dims)):
        Zg, Yg, smp = ts.leverage_sketch(Tg, n, Ag, m, seed=5, sweep=3)
        Zw, Yw, sw, _ = sketch.leverage_sketch_dense(T, n, A, m, seed=5, sweep=3)
        assert np.array_equal(smp.cpu().numpy(), sw)
        assert np.allclose(Zg.cpu().numpy(), Zw, rtol=1e-13, atol=0)
        assert np.allclose(Yg.cpu().numpy(), Yw, rtol=1e-13, atol=0)


def _coo_dup(dims, nnz, seed, zipf=False):
    g = np.random.default_rng(seed)
    if zipf:
        idx = np.stack([np.minimum(np.searchsorted(synth.zipf_table(s, 1.1), g.random(nnz),
                                                   side="right"), s - 1) for s in dims])
    else:
        idx = np.stack([g.integers(0, s, nnz) for s in dims])
    idx = idx.astype(np.int32)
    idx[:, nnz // 2:nnz // 2 + 7] = idx[:, :7]     # repeated coordinates
    return idx, g.standard_normal(nnz)


@pytest.mark.parametrize("dims,nnz,m,zipf", [((40, 30, 20), 3000, 400, False),
                                             ((12, 10, 9, 8), 2000, 150, False),
                                             ((3000, 2000, 1500), 200000, 1000, True)])
@pytest.mark.parametrize("det", [False, True])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_leverage_coo_sketch_matches_oracle(ts, dims, nnz, m, zipf, det, dtype):
    # COO leverage sketch through the fibre index: the same multi-indices as the oracle
    # (bit-exact), Y rows gathered from the nonzeros of the sampled fibres (empty
    # fibres give zero rows; repeated coordinates add)
    if det and zipf:
        pytest.skip("deterministic selection scores all 3e6 candidates: covered by the dense test")
    idx, vals = _coo_dup(dims, nnz, seed=6, zipf=zipf)
    if dtype == torch.float32:
        vals = vals.astype(np.float32).astype(np.float64)
    g = np.random.default_rng(7)
    R = 3
    fac = [np.linalg.qr(g.standard_normal((s, R)))[0] for s in dims]
    if dtype == torch.float32:
        fac = [f.astype(np.float32).astype(np.float64) for f in fac]
    X = ts.Coo(torch.from_numpy(idx).cuda().contiguous(), dev(vals, dtype), tuple(dims))
    Ag = [dev(f, dtype) for f in fac]
    tol = 1e-13 if dtype == torch.float64 else 1e-5
    for n in range(len(dims)):
        if det:
            Zw, Yw, sw = sketch.leverage_sketch_coo_det(idx, vals, dims, n, fac, m)
            Zg, Yg, sg = ts.leverage_sketch_det(X, n, Ag, m)
        else:
            Zw, Yw, sw, _ = sketch.leverage_sketch_coo(idx, vals, dims, n, fac, m, 5, 2)
            Zg, Yg, sg = ts.leverage_sketch(X, n, Ag, m, seed=5, sweep=2)
        nsel = sw.shape[0]
        assert np.array_equal(sg.cpu().numpy()[:nsel], sw.astype(np.int32))
        Zg, Yg = Zg.double().cpu().numpy(), Yg.double().cpu().numpy()
        assert np.abs(Zg[:nsel] - Zw).max() <= tol * max(1.0, np.abs(Zw).max())
        assert np.abs(Yg[:nsel] - Yw).max() <= tol * max(1.0, np.abs(Yw).max())
        assert np.count_nonzero(Yw) > 0
        if zipf:
            assert (np.abs(Yw).sum(axis=1) == 0).any()  # sampled fibres holding no nonzero


# ---------------------------------------------------------------- a9 fitness

@pytest.mark.parametrize("dims,ranks,dtype", [((40, 40, 40), (5, 5, 5), torch.float64),
                                              ((400, 400, 400), (10, 10, 10), torch.float32),
                                              ((30, 20, 25, 10), (3, 2, 4, 2), torch.float64),
                                              ((123, 77), (6, 5), torch.float32)])
def test_fitness_matches_direct_reconstruction(ts, dims, ranks, dtype):
    T, core, A = synth.dense_tucker(dims, ranks, 1e-2, seed=9,
                                    dtype=np.float64 if dtype == torch.float64 else np.float32)
    core = core * 1.01        # a model that is not the exact projection
    Tx = T.astype(np.float64)
    coreg = dev(core, dtype)
    Ag = [dev(a, dtype) for a in A]
    if dtype == torch.float32:
        core = coreg.double().cpu().numpy()
        A = [a.double().cpu().numpy() for a in Ag]
    want = tucker.residual(Tx, core, A)
    got = ts.fitness_residual(dev(T), coreg, Ag)
    tol = 1e-12 if dtype == torch.float64 else 1e-5
    assert abs(got - want) <= tol * want


@pytest.mark.parametrize("dims,ranks,nnz,dtype", [((40, 30, 20), (5, 4, 3), 5000, torch.float64),
                                                   ((40, 30, 20), (5, 4, 3), 5000, torch.float32),
                                                   ((30, 20, 25, 10), (3, 2, 4, 2), 8000,
                                                    torch.float64),
                                                   ((3000, 2000, 1500), (8, 8, 8), 300000,
                                                    torch.float32),
                                                   ((20, 25, 30), (3, 4, 20), 3000, torch.float64),
                                                   ((9, 8, 7, 6, 5), (2, 3, 2, 3, 2), 2000,
                                                    torch.float64),
                                                   ((50, 40), (12, 9), 1500, torch.float32)])
def test_fitness_coo_matches_oracle(ts, dims, ranks, nnz, dtype):
    # ||T||^2 - 2 <T, T~> + ||T~||^2 with repeated coordinates merged for ||T||^2, against
    # the oracle's identity (itself pinned to direct reconstruction); factors not
    # orthonormal, so ||T~|| is not ||C||.  Shapes cover the unrolled order-2/3/4 forms
    # and the general one (a rank above 16, order 5).
    idx, vals = _coo_dup(dims, nnz, seed=8, zipf=dims[0] > 1000)
    g = np.random.default_rng(9)
    core = g.standard_normal(ranks)
    A = [g.standard_normal((s, R)) / np.sqrt(s) for s, R in zip(dims, ranks)]
    if dtype == torch.float32:
        vals = vals.astype(np.float32).astype(np.float64)
        core = core.astype(np.float32).astype(np.float64)
        A = [a.astype(np.float32).astype(np.float64) for a in A]
    want = tucker.residual(tucker.Coo(idx.astype(np.int64), vals, dims), core, A)
    X = ts.Coo(torch.from_numpy(idx).cuda().contiguous(), dev(vals, dtype), tuple(dims))
    got = ts.fitness_residual(X, dev(core, dtype), [dev(a, dtype) for a in A])
    tol = 1e-11 if dtype == torch.float64 else 1e-5
    assert abs(got - want) <= tol * max(want, 1e-3)


def test_coo_empty_tensor(ts):
    # nnz = 0: the leverage sketch has zero right-hand sides (Z is still the sampled rows
    # of the Kronecker product) and the residual of the empty tensor is reported as 0,
    # as in the dense form
    dims = (12, 10, 9)
    g = np.random.default_rng(3)
    fac = [np.linalg.qr(g.standard_normal((s, 3)))[0] for s in dims]
    X = ts.Coo(torch.zeros((3, 0), dtype=torch.int32, device="cuda"),
               torch.zeros(0, dtype=torch.float64, device="cuda"), dims)
    Zg, Yg, sg = ts.leverage_sketch(X, 1, [dev(f) for f in fac], 50, seed=2, sweep=0)
    Zw, Yw, sw, _ = sketch.leverage_sketch_coo(np.zeros((3, 0), np.int32), np.zeros(0), dims, 1,
                                               fac, 50, 2, 0)
    assert np.array_equal(sg.cpu().numpy(), sw.astype(np.int32))
    assert np.allclose(Zg.cpu().numpy(), Zw, rtol=1e-13, atol=0)
    assert not Yg.cpu().numpy().any() and not Yw.any()
    core = g.standard_normal((3, 3, 3))
    assert ts.fitness_residual(X, dev(core), [dev(f) for f in fac]) == 0.0


def test_fitness_coo_exact_model_is_zero(ts):
    # a COO tensor holding every entry of a Tucker tensor once (plus explicit repeats
    # that cancel) has residual ~0 against its own model
    dims, ranks = (12, 9, 7), (3, 2, 2)
    T, core, A = synth.dense_tucker(dims, ranks, 0.0, seed=10)
    idx = np.stack(np.unravel_index(np.arange(T.size), dims)).astype(np.int32)
    vals = T.reshape(-1)
    idx = np.concatenate([idx, idx[:, :50], idx[:, :50]], axis=1)
    vals = np.concatenate([vals, np.full(50, 0.25), np.full(50, -0.25)])
    X = ts.Coo(torch.from_numpy(idx).cuda().contiguous(), dev(vals), dims)
    got = ts.fitness_residual(X, dev(core), [dev(a) for a in A])
    assert got < 1e-6   # sqrt of a cancellation at FP64 rounding


# ---------------------------------------------------------------- a7/a10 BF16 Gram products

def _bf16_round(x):
    """Round FP32 values to BF16 (nearest, ties to even), returned as FP32."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("M,N,K", [(100, 515, 2000), (37, 70, 100), (128, 256, 64),
                                   (200, 300, 1000), (1, 1, 1), (130, 129, 65)])
def test_gram_bf16_matches_rounded_product(ts, M, N, K):
    g = np.random.default_rng(M * 7 + N + K)
    A = g.standard_normal((M, K)).astype(np.float32)
    B = g.standard_normal((N, K)).astype(np.float32)
    C = ts.gram_bf16(dev(A, torch.float32), dev(B, torch.float32)).cpu().numpy()
    want = _bf16_round(A).astype(np.float64) @ _bf16_round(B).astype(np.float64).T
    # products of BF16 values are exact in FP32: only the FP32 accumulation differs
    scale = np.sqrt(K) * np.abs(_bf16_round(A)).max() * np.abs(_bf16_round(B)).max()
    assert np.max(np.abs(C - want)) <= 4e-6 * scale
    # and the rounding of the operands is what separates it from the FP64 product
    exact = A.astype(np.float64) @ B.astype(np.float64).T
    assert np.max(np.abs(C - exact)) <= 2e-2 * scale
