// Gradient of the sketched fit of one subproblem (the objective each step of Alg. 4
// minimises, eq. (tucker_ls) with the TensorSketch of Sec. 3.1 on the left):
//   L = 1/2 || Z C_(n)^T A^(n)T - Y ||_F^2,   Z = TensorSketch of the factors k != n.
// With M = C_(n)^T A^(n)T and R = Z M - Y:
//   dL/dA^(n) = (Z^T R)^T C_(n)^T,   dL/dC_(n) = (Z^T R A^(n))^T,   dL/dZ = R M^T,
// and dL/dZ flows to the factors k != n through the adjoint of the FFT chain and the
// transpose of each CountSketch (launch_ts_adjoint).  Everything runs on the caller's
// stream in the caller's scratch.
#include "internal.cuh"

namespace ts {

namespace {

// Multi-index of element e of a C-order tensor with `order` modes of extents `dims`.
struct Unfolding {
  int order, n;
  int dims[TS_MAX_ORDER];
};

// The mode-n unfolding column of core element e and its mode-n index.
__device__ __forceinline__ void unfold_index(const Unfolding& u, long e, int* row, long* col) {
  long rem = e, c = 0, stride = 1;
  int a = 0;
  for (int k = u.order - 1; k >= 0; --k) {
    const int ik = (int)(rem % u.dims[k]);
    rem /= u.dims[k];
    if (k == u.n) {
      a = ik;
    } else {
      c += ik * stride;
      stride *= u.dims[k];
    }
  }
  *row = a;
  *col = c;
}

// Cn (R_n x r, row-major) = the mode-n unfolding of the core.
template <typename T>
__global__ void k_unfold(Unfolding u, long total, long r, const T* __restrict__ core,
                         T* __restrict__ Cn) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    int a;
    long c;
    unfold_index(u, e, &a, &c);
    Cn[a * r + c] = core[e];
  }
}

// grad_core[e] = dCnT[c, a] for the unfolding position (a, c) of element e (dCnT: r x R_n).
template <typename T>
__global__ void k_fold_transposed(Unfolding u, long total, int Rn, const T* __restrict__ dCnT,
                                  T* __restrict__ grad_core) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    int a;
    long c;
    unfold_index(u, e, &a, &c);
    grad_core[e] = dCnT[c * Rn + a];
  }
}

// *out = 1/2 sum x^2, accumulated in FP64 (out zeroed by the caller).
template <typename T>
__global__ void k_half_sumsq(long n, const T* __restrict__ x, double* __restrict__ out) {
  double s = 0;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x) {
    const double v = (double)x[e];
    s += v * v;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) atomicAdd(out, 0.5 * s);
  }
}

struct GradShape {
  int N, n, m;
  int64_t dims[TS_MAX_ORDER];
  int ranks[TS_MAX_ORDER];
  long r, core_elems, s;
  int cols_sum;
};

template <typename T>
struct GradWork {
  Cx<T>* tw;
  Cx<T>* spectra;
  T *Z, *Cn, *M, *R, *W, *dZ, *dU, *dCnT;
  Cx<T>* dspec;
};

template <typename T>
void grad_carve(const GradShape& g, Bump& b, GradWork<T>& w) {
  const size_t m = g.m;
  w.tw = b.take<Cx<T>>(m);
  w.spectra = b.take<Cx<T>>(m * g.cols_sum);
  w.Z = b.take<T>(m * g.r);
  w.Cn = b.take<T>((size_t)g.core_elems);
  w.M = b.take<T>((size_t)g.r * g.s);
  w.R = b.take<T>(m * g.s);
  w.W = b.take<T>((size_t)g.r * g.s);
  w.dZ = b.take<T>(m * g.r);
  w.dspec = b.take<Cx<T>>(m * g.r);
  w.dU = b.take<T>(m * g.cols_sum);
  w.dCnT = b.take<T>((size_t)g.core_elems);
}

template <typename T>
MatView<T> view(const T* p, long rs, long cs) {
  return MatView<T>{p, rs, cs};
}
template <typename T>
OutView<T> oview(T* p, long rs, long cs) {
  return OutView<T>{p, rs, cs};
}

template <typename T>
ts_status fit_grad_impl(const GradShape& g, const T* core, const T* const* A,
                        const int32_t* const* tables, const T* Y, double* loss, T* grad_core,
                        T* const* grad_A, GradWork<T>& w, cudaStream_t st) {
  const int N = g.N, n = g.n, m = g.m, Rn = g.ranks[n];
  const long r = g.r, s = g.s;
  const T* chain[TS_MAX_ORDER];
  const int32_t* ctab[TS_MAX_ORDER];
  int64_t rows[TS_MAX_ORDER];
  int cols[TS_MAX_ORDER];
  T* gchain[TS_MAX_ORDER];
  int nf = 0;
  for (int k = 0; k < N; ++k)
    if (k != n) {
      chain[nf] = A[k];
      ctab[nf] = tables[k];
      rows[nf] = g.dims[k];
      cols[nf] = g.ranks[k];
      gchain[nf] = grad_A ? grad_A[k] : nullptr;
      ++nf;
    }
  // Z = S P (and the factor spectra, kept for the adjoint)
  TS_TRY(launch_twiddles<T>(m, w.tw, st));
  TS_TRY(launch_ts_apply<T>(nf, chain, rows, cols, ctab, m, w.tw, w.spectra, w.Z, st));
  Unfolding u{};
  u.order = N;
  u.n = n;
  for (int k = 0; k < N; ++k) u.dims[k] = g.ranks[k];
  const int blocks = (int)std::min<long>(1024, (g.core_elems + 255) / 256);
  k_unfold<T><<<blocks, 256, 0, st>>>(u, g.core_elems, r, core, w.Cn);
  TS_LAUNCH_CHECK();
  // M = C_(n)^T A^(n)T (r x s)
  TS_TRY(gemm<T>((int)r, (int)s, Rn, 1.0, view<T>(w.Cn, 1, r), view<T>(A[n], 1, Rn), 0.0,
                 oview<T>(w.M, s, 1), nullptr, st));
  // R = Z M - Y (m x s)
  TS_CUDA(cudaMemcpyAsync(w.R, Y, sizeof(T) * (size_t)m * s, cudaMemcpyDeviceToDevice, st));
  TS_TRY(gemm<T>(m, (int)s, (int)r, 1.0, view<T>(w.Z, 1, m), view<T>(w.M, s, 1), -1.0,
                 oview<T>(w.R, s, 1), nullptr, st));
  TS_CUDA(cudaMemsetAsync(loss, 0, sizeof(double), st));
  k_half_sumsq<T><<<(int)std::min<long>(1024, ((long)m * s + 255) / 256), 256, 0, st>>>(
      (long)m * s, w.R, loss);
  TS_LAUNCH_CHECK();
  if (!grad_core) return TS_OK;  // the loss alone
  // W = Z^T R (r x s);  dA^(n) = W^T C_(n)^T;  dC_(n)^T = W A^(n)
  TS_TRY(gemm<T>((int)r, (int)s, m, 1.0, view<T>(w.Z, m, 1), view<T>(w.R, s, 1), 0.0,
                 oview<T>(w.W, s, 1), nullptr, st));
  TS_TRY(gemm<T>((int)s, Rn, (int)r, 1.0, view<T>(w.W, 1, s), view<T>(w.Cn, 1, r), 0.0,
                 oview<T>(grad_A[n], Rn, 1), nullptr, st));
  TS_TRY(gemm<T>((int)r, Rn, (int)s, 1.0, view<T>(w.W, s, 1), view<T>(A[n], Rn, 1), 0.0,
                 oview<T>(w.dCnT, Rn, 1), nullptr, st));
  k_fold_transposed<T><<<blocks, 256, 0, st>>>(u, g.core_elems, Rn, w.dCnT, grad_core);
  TS_LAUNCH_CHECK();
  // dZ = R M^T (column-major m x r), then the chain's adjoint
  TS_TRY(gemm<T>(m, (int)r, (int)s, 1.0, view<T>(w.R, s, 1), view<T>(w.M, 1, s), 0.0,
                 oview<T>(w.dZ, 1, m), nullptr, st));
  return launch_ts_adjoint<T>(nf, rows, cols, ctab, m, w.tw, w.spectra, w.dZ, w.dspec, w.dU,
                              gchain, st);
}

ts_status grad_shape(int32_t order, const int64_t* dims, const int32_t* ranks, int32_t mode,
                     int32_t m, int32_t dtype, GradShape& g) {
  if (order < 2 || order > TS_MAX_ORDER || !dims || !ranks)
    return fail(TS_ERR_SHAPE, "ts_fit_grad: order must lie in [2, %d]", TS_MAX_ORDER);
  if (mode < 0 || mode >= order) return fail(TS_ERR_SHAPE, "ts_fit_grad: mode %d out of range", mode);
  if (dtype != TS_F32 && dtype != TS_F64) return fail(TS_ERR_INVALID_ARG, "ts_fit_grad: bad dtype");
  const int fftmax = dtype == TS_F64 ? fft_max_len<double>() : fft_max_len<float>();
  if (m < 2 || m > fftmax) return fail(TS_ERR_SHAPE, "ts_fit_grad: m=%d outside [2,%d]", m, fftmax);
  g.N = order;
  g.n = mode;
  g.m = m;
  g.r = 1;
  g.core_elems = 1;
  g.cols_sum = 0;
  for (int k = 0; k < order; ++k) {
    if (dims[k] < 1 || ranks[k] < 1 || dims[k] > (1l << 31))
      return fail(TS_ERR_SHAPE, "ts_fit_grad: dims[%d]=%lld, ranks[%d]=%d", k,
                  (long long)dims[k], k, ranks[k]);
    g.dims[k] = dims[k];
    g.ranks[k] = ranks[k];
    g.core_elems *= ranks[k];
    if (k != mode) {
      g.r *= ranks[k];
      g.cols_sum += ranks[k];
    }
  }
  g.s = (long)dims[mode];
  if (g.r > (1l << 24) || (long)m * g.r > (1l << 31))
    return fail(TS_ERR_SHAPE, "ts_fit_grad: Z (m x %ld) too large", g.r);
  return TS_OK;
}

}  // namespace

}  // namespace ts

using namespace ts;

extern "C" size_t ts_fit_grad_scratch_bytes(int32_t order, const int64_t* dims,
                                            const int32_t* ranks, int32_t mode, int32_t m,
                                            int32_t dtype) {
  GradShape g;
  if (grad_shape(order, dims, ranks, mode, m, dtype, g) != TS_OK) {
    clear_error();
    return 0;
  }
  Bump b;
  if (dtype == TS_F64) {
    GradWork<double> w;
    grad_carve<double>(g, b, w);
  } else {
    GradWork<float> w;
    grad_carve<float>(g, b, w);
  }
  return b.off;
}

extern "C" ts_status ts_fit_grad(int32_t order, const int64_t* dims, const int32_t* ranks,
                                 int32_t mode, int32_t m, int32_t dtype, const void* core,
                                 const void* const* factors, const int32_t* const* tables,
                                 const void* Y, double* loss, void* grad_core,
                                 void* const* grad_factors, void* scratch, size_t scratch_bytes,
                                 ts_stream stream) {
  clear_error();
  GradShape g;
  TS_TRY(grad_shape(order, dims, ranks, mode, m, dtype, g));
  if (!core || !factors || !tables || !Y || !loss)
    return fail(TS_ERR_INVALID_ARG, "ts_fit_grad: NULL argument");
  if (!grad_core != !grad_factors)
    return fail(TS_ERR_INVALID_ARG, "ts_fit_grad: grad_core and grad_factors must both be "
                                    "given or both be NULL");
  for (int k = 0; k < order; ++k) {
    if (!factors[k] || (grad_factors && !grad_factors[k]))
      return fail(TS_ERR_INVALID_ARG, "ts_fit_grad: factor %d or its gradient NULL", k);
    if (k != mode && !tables[k]) return fail(TS_ERR_INVALID_ARG, "ts_fit_grad: table %d NULL", k);
  }
  const size_t need = ts_fit_grad_scratch_bytes(order, dims, ranks, mode, m, dtype);
  if (!scratch || scratch_bytes < need || ((uintptr_t)scratch & 255))
    return fail(TS_ERR_WORKSPACE, "ts_fit_grad: need %zu bytes of 256-aligned scratch", need);
  cudaStream_t st = (cudaStream_t)stream;
  Bump b{static_cast<char*>(scratch)};
  if (dtype == TS_F64) {
    GradWork<double> w;
    grad_carve<double>(g, b, w);
    return fit_grad_impl<double>(g, static_cast<const double*>(core),
                                 reinterpret_cast<const double* const*>(factors), tables,
                                 static_cast<const double*>(Y), loss,
                                 static_cast<double*>(grad_core),
                                 reinterpret_cast<double* const*>(grad_factors), w, st);
  }
  GradWork<float> w;
  grad_carve<float>(g, b, w);
  return fit_grad_impl<float>(g, static_cast<const float*>(core),
                              reinterpret_cast<const float* const*>(factors), tables,
                              static_cast<const float*>(Y), loss, static_cast<float*>(grad_core),
                              reinterpret_cast<float* const*>(grad_factors), w, st);
}
