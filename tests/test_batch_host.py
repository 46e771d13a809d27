"""Host-side checks of the batched C ABI (argument validation and workspace sizing).
These calls validate and plan before any device work, so they run without a GPU."""

import ctypes as C

import pytest

from paper_2104_01101_gb300 import tsketch as ts


def desc(dims, fmt=ts.TS_DENSE, dtype=ts.TS_F32):
    d = ts._Tensor()
    d.order = len(dims)
    for k, s in enumerate(dims):
        d.dims[k] = s
    d.format = fmt
    d.dtype = dtype
    d.values = C.c_void_p(0x1000)  # never dereferenced by the sizing call
    d.indices = None
    d.nnz = 0
    return d


def sizing(tensors, ranks, ms, sweeps=3, **opt):
    X = (ts._Tensor * len(tensors))(*tensors)
    flat = [r for rk in ranks for r in rk]
    rk = (C.c_int32 * max(1, len(flat)))(*flat)
    m = (C.c_int32 * max(1, len(ms)))(*ms)
    o = ts._options(0, opt.get("solve", ts.SOLVE_RSVD), 5, None, None, False, False, False,
                    gram_bf16=opt.get("gram_bf16", False))
    out = C.c_size_t(0)
    st = ts.lib().ts_batch_workspace_bytes(len(tensors), X, rk, m, sweeps, C.byref(o),
                                           C.byref(out))
    return st, out.value


def single(dims, ranks, m, sweeps=3):
    d = desc(dims)
    rk = (C.c_int32 * 3)(*ranks)
    o = ts._options(0, ts.SOLVE_RSVD, 5, None, None, False, False, False)
    out = C.c_size_t(0)
    assert ts.lib().tucker_als_workspace_bytes(C.byref(d), rk, ts.TENSORSKETCH, m, sweeps,
                                               C.byref(o), C.byref(out)) == 0
    return out.value


def test_batch_workspace_covers_every_tensor():
    shapes = [((40, 50, 60), (4, 4, 4)), ((96, 33, 72), (9, 9, 9)), ((32, 32, 32), (5, 5, 5))]
    st, total = sizing([desc(d) for d, _ in shapes], [r for _, r in shapes],
                       [8 * r[0] ** 2 for _, r in shapes])
    assert st == 0
    assert total >= sum(single(d, r, 8 * r[0] ** 2) for d, r in shapes)


@pytest.mark.parametrize("case,status", [
    ("empty", 1),              # TS_ERR_INVALID_ARG
    ("bf16", 7),               # TS_ERR_UNSUPPORTED: the precision form is single-tensor
    ("coo", 7),                # dense tensors only
    ("mixed_order", 7),
    ("exact_large_r", 7),      # exact solve with r = 81 > 64: no single-block solve
    ("rank_too_large", 2),     # TS_ERR_SHAPE from the per-tensor plan
])
def test_batch_rejects(case, status):
    if case == "empty":
        st, _ = sizing([], [], [])
    elif case == "bf16":
        st, _ = sizing([desc((40, 40, 40))], [(4, 4, 4)], [128], gram_bf16=True)
    elif case == "coo":
        st, _ = sizing([desc((40, 40, 40), fmt=ts.TS_COO)], [(4, 4, 4)], [128])
    elif case == "mixed_order":
        st, _ = sizing([desc((40, 40, 40)), desc((40, 40))], [(4, 4, 4), (4, 4, 4)], [128, 128])
    elif case == "exact_large_r":
        st, _ = sizing([desc((60, 60, 60))], [(9, 9, 9)], [648], solve=ts.SOLVE_EXACT)
    else:
        st, _ = sizing([desc((40, 40, 40)), desc((8, 40, 40))], [(4, 4, 4), (8, 4, 4)],
                       [128, 128])
    assert st == status
