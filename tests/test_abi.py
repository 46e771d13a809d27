"""The C-ABI library loads on the host and exports every entry point include/tsketch.h declares."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tsketch.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s+\*?([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                       src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "return", "sizeof")))


@pytest.fixture(scope="module")
def libpath():
    from paper_2104_01101_gb300 import build
    return build.build_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ["tucker_als_sketched", "tensorsketch_apply", "tensorsketch_input",
                 "range_finder_init", "cp_via_tucker", "ts_hash_table", "ts_last_error",
                 "ts_lrls_solve", "ts_leverage_sketch", "ts_fitness"]:
        assert want in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_prototypes_cover_the_header(libpath):
    from paper_2104_01101_gb300 import tsketch
    assert set(declared_functions()) == set(tsketch.exported_symbols())


def test_host_side_validation_without_gpu(libpath):
    # Argument checks run before any CUDA call, so they work on a host without a GPU.
    from paper_2104_01101_gb300 import tsketch
    L = tsketch.lib()
    assert L.ts_hash_table(0, 1, 0, 0, 0, -5, 10, None, None) == 1
    assert b"table_out" in L.ts_last_error()
    d = tsketch._Tensor()
    d.order = 1
    assert L.tensorsketch_input(ctypes.byref(d), 0, None, 10, None, None) == 2
    assert b"order" in L.ts_last_error()
    # workspace query of an invalid problem (rank >= dimension) reports TS_ERR_SHAPE
    d.order = 3
    for k in range(3):
        d.dims[k] = 10
    d.format, d.dtype, d.values = 0, 0, 1
    rk = (ctypes.c_int32 * 3)(10, 2, 2)
    opt = tsketch._Options()
    n = ctypes.c_size_t(0)
    assert L.tucker_als_workspace_bytes(ctypes.byref(d), rk, 0, 50, 1, ctypes.byref(opt),
                                        ctypes.byref(n)) == 2
    rk = (ctypes.c_int32 * 3)(2, 2, 2)
    assert L.tucker_als_workspace_bytes(ctypes.byref(d), rk, 0, 3, 1, ctypes.byref(opt),
                                        ctypes.byref(n)) == 2      # m < prod of other ranks
    assert L.tucker_als_workspace_bytes(ctypes.byref(d), rk, 0, 50, 1, ctypes.byref(opt),
                                        ctypes.byref(n)) == 0
    assert n.value > 0


def test_lrls_scratch_query_covers_every_supported_path(libpath):
    # Host-only sizing: the on-chip block solve, the Newton-Schulz large-r path (whose FP64
    # QR variant does not fit one block) and an unsupported shape (k > 64).
    from paper_2104_01101_gb300 import tsketch
    L = tsketch.lib()
    fused = L.ts_lrls_scratch_bytes(2000, 100, 400, 10, 0, 5, 0)
    large = L.ts_lrls_scratch_bytes(3000, 625, 300, 25, 0, 5, 0)
    assert fused > 0 and large > 4 * 625 * 625
    assert L.ts_lrls_scratch_bytes(3000, 625, 300, 70, 0, 5, 0) == 0


def _coo_desc(ts, dims, nnz):
    d = ts._Tensor()
    d.order = len(dims)
    for k, s in enumerate(dims):
        d.dims[k] = s
    d.format = ts.TS_COO
    d.dtype = ts.TS_F32
    d.values, d.indices, d.nnz = 0x1000, 0x2000, nnz   # never dereferenced by the queries
    return d


def test_coo_workspace_counts_the_residual_scratch(libpath):
    # A COO decomposition asked for its residual carves a fibre index and a hash table
    # (~40 bytes per nonzero and more); the one workspace size must cover that carve.
    from paper_2104_01101_gb300 import tsketch as ts
    L = ts.lib()
    rk = (ctypes.c_int32 * 3)(4, 4, 4)
    opt = ts._options(0, ts.SOLVE_RSVD, 5, None, None, False, False, False)

    def need(nnz, kind=ts.TENSORSKETCH):
        n = ctypes.c_size_t(0)
        d = _coo_desc(ts, (300, 250, 200), nnz)
        assert L.tucker_als_workspace_bytes(ctypes.byref(d), rk, kind, 400, 2, ctypes.byref(opt),
                                            ctypes.byref(n)) == 0
        return n.value

    assert need(1_000_000) - need(100_000) >= 40 * 900_000
    # leverage sampling adds a fibre index per mode
    assert need(1_000_000, ts.LEVERAGE) - need(100_000, ts.LEVERAGE) >= 3 * 20 * 900_000
    # a workspace one byte short is refused before any work is enqueued
    d = _coo_desc(ts, (300, 250, 200), 1000)
    fac = (ctypes.c_void_p * 3)(0x10, 0x20, 0x30)
    st = L.tucker_als_sketched(ctypes.byref(d), rk, ts.TENSORSKETCH, 400, 2, ctypes.byref(opt),
                               ctypes.c_void_p(0x100000), need(1000) - 1, ctypes.c_void_p(0x40),
                               fac, ctypes.c_void_p(0x50), None)
    assert st == 3 and b"workspace" in L.ts_last_error()   # TS_ERR_WORKSPACE
