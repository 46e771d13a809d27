"""Python binding of libtsketch.so (C ABI in include/tsketch.h).

Argument marshalling only: every step of the computation runs in the library's
CUDA kernels.  PyTorch provides device memory (outputs and scratch are torch
tensors) and the stream (torch's current stream).  Importing this module does not
load the library; the first call does, and raises if it has not been built.

Tensors
-------
A dense tensor is a contiguous CUDA torch tensor (float32 or float64).  A sparse
tensor is ``Coo(indices, values, dims)`` with ``indices`` an int32 CUDA tensor of
shape (N, nnz) and ``values`` a float32/float64 CUDA tensor of nnz entries;
repeated coordinates add.
"""

from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtsketch.so")
MAX_ORDER = 8

TS_F32, TS_F64 = 0, 1
TS_DENSE, TS_COO = 0, 1
TENSORSKETCH, LEVERAGE, LEVERAGE_DET = 0, 1, 2
SOLVE_RSVD, SOLVE_EXACT = 0, 1
PURPOSE_TS_HASH, PURPOSE_RRF_HASH, PURPOSE_RRF_GAUSS, PURPOSE_RSVD_GAUSS, PURPOSE_LEV_UNIFORM = 1, 2, 3, 4, 5

_STATUS = {0: "TS_OK", 1: "TS_ERR_INVALID_ARG", 2: "TS_ERR_SHAPE", 3: "TS_ERR_WORKSPACE",
           4: "TS_ERR_CUDA", 5: "TS_ERR_TIMEOUT", 6: "TS_ERR_NUMERIC", 7: "TS_ERR_UNSUPPORTED"}


class TsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Tensor(C.Structure):
    _fields_ = [("order", C.c_int32), ("dims", C.c_int64 * MAX_ORDER), ("format", C.c_int32),
                ("dtype", C.c_int32), ("values", C.c_void_p), ("indices", C.c_void_p),
                ("nnz", C.c_int64)]


class _Options(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("rrf_k1", C.c_int32), ("rrf_k2", C.c_int32),
                ("rsvd_oversample", C.c_int32), ("solve", C.c_int32),
                ("resketch_each_sweep", C.c_int32), ("gram_bf16", C.c_int32),
                ("init_given", C.c_int32), ("track_fit", C.c_int32),
                ("solve_fp64", C.c_int32), ("use_graph", C.c_int32),
                ("phase_events", C.POINTER(C.c_void_p))]


_lib = None
P = C.c_void_p
PP = C.POINTER(C.c_void_p)
I32, I64, U64, SZ = C.c_int32, C.c_int64, C.c_uint64, C.c_size_t
TP = C.POINTER(_Tensor)
OP = C.POINTER(_Options)

_PROTOS = {
    "ts_last_error": (C.c_char_p, []),
    "ts_version": (C.c_char_p, []),
    "ts_kernel_launches": (C.c_uint64, []),
    "ts_hash_table": (I32, [U64, I32, I32, I32, I32, I64, I32, P, P]),
    "tensorsketch_apply_scratch_bytes": (SZ, [I32, C.POINTER(I32), I32, I32]),
    "tensorsketch_apply": (I32, [I32, PP, C.POINTER(I64), C.POINTER(I32), PP, I32, I32, P, P, SZ, P]),
    "tensorsketch_apply_static_scratch_capacity": (SZ, []),
    "tensorsketch_apply_static_scratch": (I32, [I32, PP, C.POINTER(I64), C.POINTER(I32), PP, I32,
                                                I32, P, P]),
    "tensorsketch_input": (I32, [TP, I32, PP, I32, P, P]),
    "range_finder_init_scratch_bytes": (SZ, [TP, I32, I32, I32, I32]),
    "range_finder_init": (I32, [TP, I32, I32, I32, I32, U64, P, P, SZ, P]),
    "ts_gram_bf16_scratch_bytes": (SZ, [I32, I32, I32]),
    "ts_gram_bf16": (I32, [I32, I32, I32, P, P, P, P, SZ, P]),
    "ts_lrls_scratch_bytes": (SZ, [I32, I32, I32, I32, I32, I32, I32]),
    "ts_lrls_solve": (I32, [I32, I32, I32, I32, I32, P, P, I32, U64, I32, I32, I32, I32, P, P, P,
                            SZ, P]),
    "ts_leverage_sketch_scratch_bytes": (SZ, [TP, I32, I32]),
    "ts_leverage_sketch": (I32, [TP, I32, C.POINTER(I32), PP, I32, U64, I32, P, P, P, P, SZ, P]),
    "ts_leverage_sketch_det": (I32, [TP, I32, C.POINTER(I32), PP, I32, P, P, P, P, SZ, P]),
    "ts_fitness_scratch_bytes": (SZ, [TP, C.POINTER(I32)]),
    "ts_fitness": (I32, [TP, C.POINTER(I32), P, PP, P, P, SZ, P]),
    "tucker_als_workspace_bytes": (I32, [TP, C.POINTER(I32), I32, I32, I32, OP, C.POINTER(SZ)]),
    "tucker_als_sketched": (I32, [TP, C.POINTER(I32), I32, I32, I32, OP, P, SZ, P, PP, P, P]),
    "cp_via_tucker_workspace_bytes": (I32, [TP, I32, C.POINTER(I32), I32, I32, OP, C.POINTER(SZ)]),
    "cp_via_tucker": (I32, [TP, I32, C.POINTER(I32), I32, I32, I32, OP, P, SZ, PP, P, P]),
    "ts_cp_als_scratch_bytes": (SZ, [I32, C.POINTER(I32), I32, I32]),
    "ts_cp_als": (I32, [I32, C.POINTER(I32), I32, I32, I32, P, PP, P, SZ, P]),
    "ts_fit_grad_scratch_bytes": (SZ, [I32, C.POINTER(I64), C.POINTER(I32), I32, I32, I32]),
    "ts_fit_grad": (I32, [I32, C.POINTER(I64), C.POINTER(I32), I32, I32, I32, P, PP, PP, P, P, P,
                          PP, P, SZ, P]),
    "ts_batch_workspace_bytes": (I32, [I32, TP, C.POINTER(I32), C.POINTER(I32), I32, OP,
                                       C.POINTER(SZ)]),
    "ts_batch_prepare": (I32, [I32, TP, C.POINTER(I32), C.POINTER(I32), I32, OP, P, SZ, PP, PP,
                               C.POINTER(P), P]),
    "ts_batch_sweeps": (I32, [P, I32, I32, P]),
    "ts_batch_residuals": (I32, [P, P, P]),
    "ts_batch_flags": (I32, [P, C.POINTER(I32)]),
    "ts_batch_tiles": (I32, [P, C.POINTER(I32), C.POINTER(C.c_float)]),
    "ts_batch_destroy": (None, [P]),
}


def lib():
    """Load libtsketch.so (built in-tree); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run __graft_entry__.build() "
                               "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_PROTOS)


def _check(st: int):
    if st != 0:
        raise TsError(st, lib().ts_last_error().decode())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor):
    return C.c_void_p(t.data_ptr())


def _ptr_array(ts):
    arr = (C.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = None if t is None else t.data_ptr()
    return arr


def _dt(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return TS_F32
    if t.dtype == torch.float64:
        return TS_F64
    raise TypeError(f"unsupported dtype {t.dtype}")


@dataclass
class Coo:
    indices: torch.Tensor   # int32 (N, nnz), CUDA
    values: torch.Tensor    # float32/float64 (nnz,), CUDA
    dims: tuple

    @property
    def dtype(self):
        return self.values.dtype

    @property
    def device(self):
        return self.values.device


def _desc(X):
    d = _Tensor()
    if isinstance(X, Coo):
        assert X.indices.dtype == torch.int32 and X.indices.is_contiguous()
        assert X.values.is_contiguous() and X.indices.shape[0] == len(X.dims)
        d.order = len(X.dims)
        for k, s in enumerate(X.dims):
            d.dims[k] = int(s)
        d.format = TS_COO
        d.dtype = _dt(X.values)
        d.values = X.values.data_ptr()
        d.indices = X.indices.data_ptr()
        d.nnz = int(X.values.numel())
    else:
        if not (X.is_cuda and X.is_contiguous()):
            raise ValueError("dense tensors must be contiguous CUDA tensors")
        d.order = X.dim()
        for k, s in enumerate(X.shape):
            d.dims[k] = int(s)
        d.format = TS_DENSE
        d.dtype = _dt(X)
        d.values = X.data_ptr()
        d.indices = None
        d.nnz = 0
    return d


def _dims(X):
    return tuple(X.dims) if isinstance(X, Coo) else tuple(X.shape)


def _scratch(nbytes: int, device):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


# ---------------------------------------------------------------- entry points

def version() -> str:
    return lib().ts_version().decode()


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    return int(lib().ts_kernel_launches())


def hash_table(seed, purpose, sweep, n, k, size, nbins, device="cuda"):
    out = torch.empty(size, dtype=torch.int32, device=device)
    _check(lib().ts_hash_table(seed, purpose, sweep, n, k, size, nbins, _ptr(out), _stream()))
    return out


def tensorsketch_apply(factors, tables, m: int):
    """Z = S (F_0 (x) ... ) as an (m, prod cols) tensor (a transposed view of column-major storage)."""
    nf = len(factors)
    dt = _dt(factors[0])
    rows = (C.c_int64 * nf)(*[f.shape[0] for f in factors])
    cols = (C.c_int32 * nf)(*[f.shape[1] for f in factors])
    ncols = 1
    for f in factors:
        ncols *= f.shape[1]
    dev = factors[0].device
    Zt = torch.empty((ncols, m), dtype=factors[0].dtype, device=dev)
    nbytes = lib().tensorsketch_apply_scratch_bytes(nf, cols, m, dt)
    scr = _scratch(nbytes, dev)
    _check(lib().tensorsketch_apply(nf, _ptr_array(factors), rows, cols, _ptr_array(tables), m, dt,
                                    _ptr(Zt), _ptr(scr), scr.numel(), _stream()))
    return Zt.t()


def tensorsketch_apply_static_scratch(factors, tables, m: int):
    """As tensorsketch_apply, but the library uses its fixed device scratch array and
    nothing is allocated for scratch (only the output Z is a new tensor here)."""
    nf = len(factors)
    dt = _dt(factors[0])
    rows = (C.c_int64 * nf)(*[f.shape[0] for f in factors])
    cols = (C.c_int32 * nf)(*[f.shape[1] for f in factors])
    ncols = 1
    for f in factors:
        ncols *= f.shape[1]
    Zt = torch.empty((ncols, m), dtype=factors[0].dtype, device=factors[0].device)
    _check(lib().tensorsketch_apply_static_scratch(nf, _ptr_array(factors), rows, cols,
                                                   _ptr_array(tables), m, dt, _ptr(Zt), _stream()))
    return Zt.t()


def tensorsketch_input(X, mode: int, tables, m: int):
    dims = _dims(X)
    dtype = X.dtype
    dev = X.device
    Y = torch.empty((m, dims[mode]), dtype=dtype, device=dev)
    tabs = [tables[k] if k != mode else None for k in range(len(dims))]
    d = _desc(X)
    _check(lib().tensorsketch_input(C.byref(d), mode, _ptr_array(tabs), m, _ptr(Y), _stream()))
    return Y


def range_finder_init(X, mode: int, R: int, k1: int, k2: int, seed: int):
    dims = _dims(X)
    d = _desc(X)
    A = torch.empty((dims[mode], R), dtype=X.dtype, device=X.device)
    nbytes = lib().range_finder_init_scratch_bytes(C.byref(d), mode, R, k1, k2)
    scr = _scratch(nbytes, X.device)
    _check(lib().range_finder_init(C.byref(d), mode, R, k1, k2, seed, _ptr(A), _ptr(scr),
                                   scr.numel(), _stream()))
    return A


def gram_bf16(A, B):
    """C = bf16(A) bf16(B)^T with FP32 accumulation on the tensor cores; A (M, K) and
    B (N, K) FP32 on the device."""
    M, K = A.shape
    N = B.shape[0]
    Ac = A.contiguous()
    Bc = B.contiguous()
    Cout = torch.empty((M, N), dtype=torch.float32, device=A.device)
    scr = _scratch(lib().ts_gram_bf16_scratch_bytes(M, N, K), A.device)
    _check(lib().ts_gram_bf16(M, N, K, _ptr(Ac), _ptr(Bc), _ptr(Cout), _ptr(scr), scr.numel(),
                              _stream()))
    return Cout


def lrls_solve(Z, Y, R: int, solve: int = SOLVE_RSVD, seed: int = 0, sweep: int = 0, n: int = 0,
               oversample: int = 5, solve_fp64: bool = False):
    """Sketched rank-constrained LS; Z is (m, r) (any strides), Y is (m, s)."""
    m, r = Z.shape
    s = Y.shape[1]
    dt = _dt(Y)
    Zc = Z.t().contiguous()          # column-major storage of Z
    Yc = Y.contiguous()
    CnT = torch.empty((r, R), dtype=Y.dtype, device=Y.device)
    A = torch.empty((s, R), dtype=Y.dtype, device=Y.device)
    nbytes = lib().ts_lrls_scratch_bytes(m, r, s, R, solve, oversample, dt)
    scr = _scratch(nbytes, Y.device)
    _check(lib().ts_lrls_solve(m, r, s, R, dt, _ptr(Zc), _ptr(Yc), solve, seed, sweep, n, oversample,
                               int(solve_fp64), _ptr(CnT), _ptr(A), _ptr(scr), scr.numel(),
                               _stream()))
    return CnT, A


def _check_scratch_flag(scr):
    """The int32 at offset 0 of a leverage sketch's scratch: non-zero if the fibre index
    of a COO tensor could not place a nonzero (synchronises)."""
    if int(scr[:4].view(torch.int32).item()) != 0:
        raise TsError(6, "fibre index overflow flagged by the device")


def leverage_sketch(X, mode: int, factors, m: int, seed: int, sweep: int = 0):
    dims = _dims(X)
    N = len(dims)
    ranks = [f.shape[1] if f is not None else 1 for f in factors]
    r = 1
    for k in range(N):
        if k != mode:
            r *= ranks[k]
    d = _desc(X)
    Zt = torch.empty((r, m), dtype=X.dtype, device=X.device)
    Y = torch.empty((m, dims[mode]), dtype=X.dtype, device=X.device)
    samples = torch.empty((m, N - 1), dtype=torch.int32, device=X.device)
    nbytes = lib().ts_leverage_sketch_scratch_bytes(C.byref(d), mode, m)
    scr = _scratch(nbytes, X.device)
    rk = (C.c_int32 * N)(*ranks)
    facs = [factors[k] if k != mode else None for k in range(N)]
    _check(lib().ts_leverage_sketch(C.byref(d), mode, rk, _ptr_array(facs), m, seed, sweep,
                                    _ptr(Zt), _ptr(Y), _ptr(samples), _ptr(scr), scr.numel(),
                                    _stream()))
    _check_scratch_flag(scr)
    return Zt.t(), Y, samples


def leverage_sketch_det(X, mode: int, factors, m: int):
    """Deterministic leverage sketch (ts_leverage_sketch_det): (Z, Y, samples)."""
    dims = _dims(X)
    N = len(dims)
    ranks = [f.shape[1] if f is not None else 1 for f in factors]
    r = 1
    for k in range(N):
        if k != mode:
            r *= ranks[k]
    d = _desc(X)
    Zt = torch.empty((r, m), dtype=X.dtype, device=X.device)
    Y = torch.empty((m, dims[mode]), dtype=X.dtype, device=X.device)
    samples = torch.empty((m, N - 1), dtype=torch.int32, device=X.device)
    nbytes = lib().ts_leverage_sketch_scratch_bytes(C.byref(d), mode, m)
    scr = _scratch(nbytes, X.device)
    rk = (C.c_int32 * N)(*ranks)
    facs = [factors[k] if k != mode else None for k in range(N)]
    _check(lib().ts_leverage_sketch_det(C.byref(d), mode, rk, _ptr_array(facs), m, _ptr(Zt),
                                        _ptr(Y), _ptr(samples), _ptr(scr), scr.numel(), _stream()))
    _check_scratch_flag(scr)
    return Zt.t(), Y, samples


def fitness_residual(X, core, factors) -> float:
    """Relative residual ||T - T~|| / ||T|| (synchronises)."""
    d = _desc(X)
    N = len(factors)
    rk = (C.c_int32 * N)(*[f.shape[1] for f in factors])
    out = torch.zeros(1, dtype=torch.float64, device=core.device)
    nbytes = lib().ts_fitness_scratch_bytes(C.byref(d), rk)
    scr = _scratch(nbytes, core.device)
    _check(lib().ts_fitness(C.byref(d), rk, _ptr(core.contiguous()), _ptr_array(factors), _ptr(out),
                            _ptr(scr), scr.numel(), _stream()))
    return float(out.item())


def _options(seed, solve, oversample, rrf_k1, rrf_k2, resketch, init_given, track_fit,
             solve_fp64=False, use_graph=False, gram_bf16=False):
    o = _Options()
    o.seed = seed
    o.rrf_k1 = rrf_k1 or 0
    o.rrf_k2 = rrf_k2 or 0
    o.rsvd_oversample = oversample
    o.solve = solve
    o.resketch_each_sweep = int(bool(resketch))
    o.gram_bf16 = int(bool(gram_bf16))
    o.init_given = int(bool(init_given))
    o.track_fit = int(bool(track_fit))
    o.solve_fp64 = int(bool(solve_fp64))
    o.use_graph = int(bool(use_graph))
    return o


class TuckerPlan:
    """Reusable workspace + outputs for repeated tucker_als_sketched calls on one shape."""

    def __init__(self, X, ranks, m, sweeps, kind=TENSORSKETCH, seed=0, solve=SOLVE_RSVD,
                 oversample=5, rrf_k1=None, rrf_k2=None, resketch=False, track_fit=False,
                 want_residual=True, solve_fp64=False, use_graph=False, gram_bf16=False):
        self.dims = _dims(X)
        self.N = len(self.dims)
        self.ranks = list(ranks)
        self.kind, self.m, self.sweeps = kind, m, sweeps
        self.opt = _options(seed, solve, oversample, rrf_k1, rrf_k2, resketch, False, track_fit,
                            solve_fp64, use_graph, gram_bf16)
        self.track_fit = track_fit
        self.want_residual = want_residual
        dtype, dev = X.dtype, X.device
        d = _desc(X)
        self._rk = (C.c_int32 * self.N)(*self.ranks)
        nbytes = C.c_size_t(0)
        _check(lib().tucker_als_workspace_bytes(C.byref(d), self._rk, kind, m, sweeps,
                                                C.byref(self.opt), C.byref(nbytes)))
        self.workspace = _scratch(nbytes.value, dev)
        self.core = torch.zeros(self.ranks, dtype=dtype, device=dev)
        self.factors = [torch.zeros((s, R), dtype=dtype, device=dev)
                        for s, R in zip(self.dims, self.ranks)]
        self.residuals = torch.zeros(max(sweeps, 1), dtype=torch.float64, device=dev)

    def set_phase_events(self, events):
        """Record the 6 phase events of the driver (torch.cuda.Event list) on every run."""
        self._events = events
        for e in events or []:
            e.record()          # torch creates the CUDA event lazily, on first record
        torch.cuda.synchronize()
        self._ev_arr = (C.c_void_p * 6)(*[e.cuda_event for e in events]) if events else None
        self.opt.phase_events = (C.cast(self._ev_arr, C.POINTER(C.c_void_p))
                                 if events else None)

    def run(self, X, init_factors=None):
        """Enqueue one decomposition on the current stream (no synchronisation)."""
        d = _desc(X)
        self.opt.init_given = 0
        if init_factors is not None:
            for k, a in enumerate(init_factors):
                if a is not None:
                    self.factors[k].copy_(a)
            self.opt.init_given = 1
        res = _ptr(self.residuals) if self.want_residual else None
        _check(lib().tucker_als_sketched(C.byref(d), self._rk, self.kind, self.m, self.sweeps,
                                         C.byref(self.opt), _ptr(self.workspace),
                                         self.workspace.numel(), _ptr(self.core),
                                         _ptr_array(self.factors), res, _stream()))
        return self

    def numeric_flag(self) -> int:
        return int(self.workspace[:4].view(torch.int32).item())


def fit_grad(core, factors, Y, tables, mode: int, m: int, want_grad: bool = True):
    """Sketched fit of subproblem ``mode`` and its gradient (ts_fit_grad):
    returns (loss float64 0-dim tensor, grad_core, [grad of every factor]); with
    ``want_grad=False`` only the loss is computed (the gradients are None).
    ``tables``: one packed int32 device table per mode (the entry of ``mode`` is ignored,
    may be None)."""
    N = len(factors)
    dims = (C.c_int64 * N)(*[f.shape[0] for f in factors])
    rk = (C.c_int32 * N)(*[f.shape[1] for f in factors])
    dtype = _dt(core)
    nbytes = lib().ts_fit_grad_scratch_bytes(N, dims, rk, mode, m, dtype)
    if nbytes == 0:
        raise TsError(2, "ts_fit_grad: invalid shape")
    scr = _scratch(nbytes, core.device)
    core = core.contiguous()
    factors = [f.contiguous() for f in factors]
    Y = Y.contiguous()
    loss = torch.zeros((), dtype=torch.float64, device=core.device)
    gcore = torch.empty_like(core) if want_grad else None
    gfac = [torch.empty_like(f) for f in factors] if want_grad else None
    tabs = [t if t is not None else factors[0] for t in tables]  # mode's entry ignored
    _check(lib().ts_fit_grad(N, dims, rk, mode, m, dtype, _ptr(core), _ptr_array(factors),
                             _ptr_array(tabs), _ptr(Y), _ptr(loss),
                             _ptr(gcore) if want_grad else None,
                             _ptr_array(gfac) if want_grad else None, _ptr(scr), scr.numel(),
                             _stream()))
    return loss, gcore, gfac


class SketchedFit(torch.autograd.Function):
    """L = 1/2 ||Z C_(n)^T A^(n)T - Y||^2 as a differentiable function of the core and the
    factors; forward computes the loss and every gradient in one library call, backward
    scales them by the incoming gradient."""

    @staticmethod
    def forward(ctx, Y, tables, mode, m, core, *factors):
        want = any(ctx.needs_input_grad[4:])  # the gradients only when autograd needs them
        loss, gcore, gfac = fit_grad(core, list(factors), Y, tables, mode, m, want_grad=want)
        if want:
            ctx.save_for_backward(gcore, *gfac)
        return loss.to(core.dtype)

    @staticmethod
    def backward(ctx, g):
        gcore, *gfac = ctx.saved_tensors
        return (None, None, None, None, g * gcore, *[g * x for x in gfac])


def sketched_fit(core, factors, Y, tables, mode: int, m: int):
    """Differentiable sketched fit (see SketchedFit)."""
    return SketchedFit.apply(Y, tables, mode, m, core, *factors)


class TuckerBatch:
    """Batched Sketch-Tucker-ALS of many dense tensors (ts_batch_* in the C ABI).

    ``tensors``: list of contiguous CUDA tensors of one order and dtype; ``ranks``: one
    rank tuple per tensor; ``ms``: one sketch size per tensor.  Tensor i uses seed
    ``seed + i``.  Construction runs the one-time setup (and the tile autotuner) and
    synchronises; ``sweeps(first, n)`` enqueues sweeps [first, first + n) of every
    tensor on the current stream (capturable in a CUDA graph)."""

    def __init__(self, tensors, ranks, ms, sweeps, seed=0, solve=SOLVE_RSVD, oversample=5,
                 rrf_k1=None, rrf_k2=None, solve_fp64=False):
        self.count = len(tensors)
        self.N = tensors[0].dim()
        self.sweeps_total = sweeps
        self.tensors = tensors  # kept alive: the batch reads them
        self.opt = _options(seed, solve, oversample, rrf_k1, rrf_k2, False, False, False,
                            solve_fp64)
        self._X = (_Tensor * self.count)(*[_desc(t) for t in tensors])
        flat = [int(r) for rk in ranks for r in rk]
        self._rk = (C.c_int32 * len(flat))(*flat)
        self._m = (C.c_int32 * self.count)(*[int(m) for m in ms])
        nbytes = C.c_size_t(0)
        _check(lib().ts_batch_workspace_bytes(self.count, self._X, self._rk, self._m, sweeps,
                                              C.byref(self.opt), C.byref(nbytes)))
        dev, dtype = tensors[0].device, tensors[0].dtype
        self.workspace = _scratch(nbytes.value, dev)
        self.cores = [torch.zeros(tuple(rk), dtype=dtype, device=dev) for rk in ranks]
        self.factors = [[torch.zeros((s, R), dtype=dtype, device=dev)
                         for s, R in zip(t.shape, rk)] for t, rk in zip(tensors, ranks)]
        self._cores = _ptr_array(self.cores)
        self._facs = _ptr_array([f for fs in self.factors for f in fs])
        self.residuals = torch.zeros(self.count, dtype=torch.float64, device=dev)
        h = C.c_void_p(None)
        _check(lib().ts_batch_prepare(self.count, self._X, self._rk, self._m, sweeps,
                                      C.byref(self.opt), _ptr(self.workspace),
                                      self.workspace.numel(), self._cores, self._facs,
                                      C.byref(h), _stream()))
        self._h = h

    def sweeps(self, first=0, n=None):
        n = self.sweeps_total - first if n is None else n
        _check(lib().ts_batch_sweeps(self._h, first, n, _stream()))
        return self

    def residual(self):
        _check(lib().ts_batch_residuals(self._h, _ptr(self.residuals), _stream()))
        return self.residuals

    def flags(self):
        out = (C.c_int32 * self.count)()
        _check(lib().ts_batch_flags(self._h, out))
        return list(out)

    def tiles(self):
        t = (C.c_int32 * self.N)()
        ms = (C.c_float * (2 * self.N))()
        _check(lib().ts_batch_tiles(self._h, t, ms))
        return list(t), [(ms[2 * n], ms[2 * n + 1]) for n in range(self.N)]

    def close(self):
        if self._h:
            torch.cuda.synchronize()
            lib().ts_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cp_via_tucker(X, R_cp: int, tucker_ranks, m: int, tucker_sweeps: int, cp_sweeps: int,
                  seed: int = 0, solve=SOLVE_RSVD, oversample: int = 5, rrf_k1=None, rrf_k2=None,
                  want_residual=True, solve_fp64=False):
    """Alg. 6: returns (CP factors [dims[k] x R_cp], residual float or None)."""
    dims = _dims(X)
    N = len(dims)
    opt = _options(seed, solve, oversample, rrf_k1, rrf_k2, False, False, False, solve_fp64)
    d = _desc(X)
    rk = (C.c_int32 * N)(*tucker_ranks)
    nbytes = C.c_size_t(0)
    _check(lib().cp_via_tucker_workspace_bytes(C.byref(d), R_cp, rk, m, tucker_sweeps,
                                               C.byref(opt), C.byref(nbytes)))
    ws = _scratch(nbytes.value, X.device)
    outs = [torch.empty((s, R_cp), dtype=X.dtype, device=X.device) for s in dims]
    res = torch.zeros(1, dtype=torch.float64, device=X.device)
    _check(lib().cp_via_tucker(C.byref(d), R_cp, rk, m, tucker_sweeps, cp_sweeps, C.byref(opt),
                               _ptr(ws), ws.numel(), _ptr_array(outs),
                               _ptr(res) if want_residual else None, _stream()))
    if int(ws[:4].view(torch.int32).item()) != 0:
        raise TsError(6, "numerical breakdown flagged by the device")
    return outs, (float(res.item()) if want_residual else None)


def cp_als(core, R_cp: int, sweeps: int):
    """CP-ALS on a dense core (ts_cp_als: HOSVD start, Alg. 2 sweeps): returns the factors
    [ranks[k] x R_cp]; raises TsError if a Gram system was flagged (synchronises)."""
    core = core.contiguous()
    order = core.dim()
    rk = (C.c_int32 * order)(*core.shape)
    dt = _dt(core)
    nbytes = lib().ts_cp_als_scratch_bytes(order, rk, R_cp, dt)
    if nbytes == 0:
        raise TsError(2, "ts_cp_als: invalid shape")
    scr = _scratch(nbytes, core.device)
    outs = [torch.empty((int(r), R_cp), dtype=core.dtype, device=core.device) for r in core.shape]
    _check(lib().ts_cp_als(order, rk, R_cp, sweeps, dt, _ptr(core), _ptr_array(outs), _ptr(scr),
                           scr.numel(), _stream()))
    if int(scr[:4].view(torch.int32).item()) != 0:
        raise TsError(6, "CP-ALS: Gram system not positive definite")
    return outs


def tucker_als_sketched(X, ranks, m: int, sweeps: int, kind=TENSORSKETCH, seed: int = 0,
                        solve=SOLVE_RSVD, oversample: int = 5, rrf_k1=None, rrf_k2=None,
                        resketch=False, init_factors=None, track_fit=False,
                        want_residual=True, solve_fp64=False, gram_bf16=False):
    """Alg. 4.  Returns (core, factors, residuals tensor or None); raises TsError on breakdown."""
    plan = TuckerPlan(X, ranks, m, sweeps, kind, seed, solve, oversample, rrf_k1, rrf_k2, resketch,
                      track_fit, want_residual, solve_fp64, gram_bf16=gram_bf16)
    plan.run(X, init_factors)
    if plan.numeric_flag() != 0:
        raise TsError(6, "numerical breakdown flagged by the device (Z^T Z not positive definite "
                         "or a non-finite eigenvalue)")
    res = None
    if want_residual:
        res = plan.residuals[:sweeps] if track_fit else plan.residuals[:1]
    return plan.core, plan.factors, res
