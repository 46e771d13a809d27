// CP-ALS on the Tucker core (Alg. 2 applied inside Alg. 6).  The core has only
// prod R_n entries, so each kernel here is a small one-shot map; the normal
// equations of every mode update use the Khatri-Rao product of the other factors
// (first factor slowest, Sec. 2.1) and the Hadamard product of their Grams.
#include "internal.cuh"

namespace ts {

struct CoreDims {
  int order;
  int ranks[TS_MAX_ORDER];
};

template <typename T>
struct FacPtrs {
  const T* p[TS_MAX_ORDER];
};

// out (R_n x prod_{k != n} R_k) = mode-n unfolding of the C-order core.
template <typename T>
__global__ void k_unfold(CoreDims d, int n, const T* __restrict__ C, T* __restrict__ out) {
  long total = 1;
  for (int k = 0; k < d.order; ++k) total *= d.ranks[k];
  const long K = total / d.ranks[n];
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    long x = e, col = 0, stride = 1;
    int row = 0;
    for (int k = d.order - 1; k >= 0; --k) {
      const int rk = (int)(x % d.ranks[k]);
      x /= d.ranks[k];
      if (k == n) {
        row = rk;
      } else {
        col += rk * stride;
        stride *= d.ranks[k];
      }
    }
    out[row * K + col] = C[e];
  }
}

// KR (prod_{k != n} R_k x Rc): row (r_k)_{k != n} in C order, column c:
// prod_k A_k(r_k, c).
template <typename T>
__global__ void k_khatri_rao(CoreDims d, int n, int Rc, FacPtrs<T> A,
                             T* __restrict__ KR) {
  long K = 1;
  for (int k = 0; k < d.order; ++k)
    if (k != n) K *= d.ranks[k];
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < K * Rc;
       e += (long)gridDim.x * blockDim.x) {
    const long row = e / Rc;
    const int c = (int)(e % Rc);
    long x = row;
    T v = 1;
    for (int k = d.order - 1; k >= 0; --k) {
      if (k == n) continue;
      const int rk = (int)(x % d.ranks[k]);
      x /= d.ranks[k];
      v *= A.p[k][rk * Rc + c];
    }
    KR[e] = v;
  }
}

// Gam (Rc x Rc) = Hadamard product over k != n of A_k^T A_k.
template <typename T>
__global__ void k_gram_hadamard(CoreDims d, int n, int Rc, FacPtrs<T> A,
                                T* __restrict__ Gam) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Rc * Rc; e += gridDim.x * blockDim.x) {
    const int a = e / Rc, b = e % Rc;
    T v = 1;
    for (int k = 0; k < d.order; ++k) {
      if (k == n) continue;
      T g = 0;
      for (int i = 0; i < d.ranks[k]; ++i) g += A.p[k][i * Rc + a] * A.p[k][i * Rc + b];
      v *= g;
    }
    Gam[e] = v;
  }
}

// One CP-ALS factor update A_n = M Gam^{-1} (M = MTTKRP, R_n x Rc) in one block, with
// Gam = Hadamard product of the other factors' Grams formed and Cholesky-factored in
// FP64: with collinear factors Gam is ill-conditioned, and the update is tiny.
template <typename T>
__global__ void __launch_bounds__(256) k_cp_update(CoreDims d, int n, int Rc, FacPtrs<T> A,
                                                   const T* __restrict__ M, T* __restrict__ out,
                                                   int* flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* L = reinterpret_cast<double*>(smem_raw);  // Rc x Rc
  double* X = L + Rc * Rc;                           // R_n x Rc (rows solved in place)
  const int Rn = d.ranks[n];
  for (int e = threadIdx.x; e < Rc * Rc; e += blockDim.x) {
    const int a = e / Rc, b = e % Rc;
    double v = 1.0;
    for (int k = 0; k < d.order; ++k) {
      if (k == n) continue;
      double g = 0.0;
      for (int i = 0; i < d.ranks[k]; ++i)
        g += (double)A.p[k][i * Rc + a] * (double)A.p[k][i * Rc + b];
      v *= g;
    }
    L[e] = v;
  }
  for (int e = threadIdx.x; e < Rn * Rc; e += blockDim.x) X[e] = (double)M[e];
  __syncthreads();
  for (int j = 0; j < Rc; ++j) {  // right-looking Cholesky, lower triangle
    if (threadIdx.x == 0) {
      double dj = L[j * Rc + j];
      if (!(dj > 0.0)) {
        if (flag) atomicExch(flag, 1);
        dj = 1.0;
      }
      L[j * Rc + j] = sqrt(dj);
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < Rc; i += blockDim.x) L[i * Rc + j] /= L[j * Rc + j];
    __syncthreads();
    for (int e = threadIdx.x; e < Rc * Rc; e += blockDim.x) {
      const int i = e / Rc, l = e % Rc;
      if (i > j && l > j && l <= i) L[i * Rc + l] -= L[i * Rc + j] * L[l * Rc + j];
    }
    __syncthreads();
  }
  // row r of A_n solves Gam x = M(r, :)^T
  for (int r = threadIdx.x; r < Rn; r += blockDim.x) {
    double* x = X + r * Rc;
    for (int i = 0; i < Rc; ++i) {
      double v = x[i];
      for (int l = 0; l < i; ++l) v -= L[i * Rc + l] * x[l];
      x[i] = v / L[i * Rc + i];
    }
    for (int i = Rc - 1; i >= 0; --i) {
      double v = x[i];
      for (int l = i + 1; l < Rc; ++l) v -= L[l * Rc + i] * x[l];
      x[i] = v / L[i * Rc + i];
    }
    for (int c = 0; c < Rc; ++c) out[r * Rc + c] = (T)x[c];
  }
}

// out (cols x rows) = in^T (in is rows x cols).
template <typename T>
__global__ void k_transpose(int rows, int cols, const T* __restrict__ in, T* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * cols; e += gridDim.x * blockDim.x)
    out[(e % cols) * rows + e / cols] = in[e];
}

// Superdiagonal core of a CP model (Rc^order entries, ones on the diagonal).
template <typename T>
__global__ void k_superdiag(int order, int Rc, T* __restrict__ D) {
  long total = 1, step = 0, p = 1;
  for (int k = 0; k < order; ++k) {
    total *= Rc;
    step += p;
    p *= Rc;
  }
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x)
    D[e] = (e % step == 0) ? (T)1 : (T)0;
}

static int grid_for(long n) {
  long b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

template <typename T>
size_t cp_core_scratch_elems(int order, const int* ranks, int Rc) {
  long total = 1, Kmax = 0;
  int Rmax = 0;
  for (int k = 0; k < order; ++k) total *= ranks[k];
  for (int n = 0; n < order; ++n) {
    const long K = total / ranks[n];
    if (K > Kmax) Kmax = K;
    if (ranks[n] > Rmax) Rmax = ranks[n];
  }
  const int E = Rmax > Rc ? Rmax : Rc;
  // unfold, KR, M, Gam, X, eigen K, partial
  return (size_t)(Rmax * Kmax + Kmax * Rc + Rmax * Rc + Rc * Rc + Rc * Rmax + E * E) +
         32 * (size_t)(Rmax * Rc > Rmax * Rmax ? Rmax * Rc : Rmax * Rmax) + 64 * 6;
}

// HOSVD initialisation (Sec. 7.2) and `sweeps` CP-ALS sweeps (Alg. 2) on the core.
// A[k] (ranks[k] x Rc) are written; scratch holds cp_core_scratch_elems<T>() values.
template <typename T>
ts_status cp_als_core(int order, const int* ranks, int Rc, int sweeps, const T* core, T* const* A,
                      T* scratch, int* flag, cudaStream_t st) {
  CoreDims d{};
  d.order = order;
  FacPtrs<T> fp{};
  for (int k = 0; k < order; ++k) fp.p[k] = A[k];
  long total = 1, Kmax = 0;
  int Rmax = 0;
  for (int k = 0; k < order; ++k) {
    d.ranks[k] = ranks[k];
    total *= ranks[k];
  }
  for (int n = 0; n < order; ++n) {
    if (total / ranks[n] > Kmax) Kmax = total / ranks[n];
    if (ranks[n] > Rmax) Rmax = ranks[n];
  }
  const int E = Rmax > Rc ? Rmax : Rc;
  T* Cn = scratch;
  T* KR = Cn + Rmax * Kmax;
  T* M = KR + Kmax * Rc;
  T* Gam = M + Rmax * Rc;
  T* X = Gam + Rc * Rc;
  T* Ke = X + Rc * Rmax;
  CoreMap none{};
  // HOSVD of the core: leading Rc eigenvectors of C_(n) C_(n)^T, canonical signs.
  for (int n = 0; n < order; ++n) {
    const long K = total / ranks[n];
    k_unfold<T><<<grid_for(total), 256, 0, st>>>(d, n, core, Cn);
    TS_LAUNCH_CHECK();
    TS_TRY(gemm<T>(ranks[n], ranks[n], (int)K, 1.0, MatView<T>{Cn, K, 1}, MatView<T>{Cn, 1, K},
                   0.0, OutView<T>{Ke, ranks[n], 1}, nullptr, st));
    TS_TRY(launch_eig_small<T>(ranks[n], Rc, Ke, nullptr, ranks[n], nullptr, nullptr, M, false,
                               flag, st));
    TS_TRY(launch_finalize<T>(ranks[n], Rc, M, Rc, 1, 0, nullptr, A[n], nullptr, 0, nullptr, none,
                              st));
  }
  for (int sweep = 0; sweep < sweeps; ++sweep) {
    for (int n = 0; n < order; ++n) {
      const long K = total / ranks[n];
      k_unfold<T><<<grid_for(total), 256, 0, st>>>(d, n, core, Cn);
      TS_LAUNCH_CHECK();
      k_khatri_rao<T><<<grid_for(K * Rc), 256, 0, st>>>(d, n, Rc, fp, KR);
      TS_LAUNCH_CHECK();
      // MTTKRP: M = C_(n) KR (R_n x Rc)
      TS_TRY(gemm<T>(ranks[n], Rc, (int)K, 1.0, MatView<T>{Cn, K, 1}, MatView<T>{KR, Rc, 1}, 0.0,
                     OutView<T>{M, Rc, 1}, nullptr, st));
      // A_n = M Gam^{-1} with Gam = *_{k != n} A_k^T A_k (FP64 normal equations)
      const size_t smem = sizeof(double) * ((size_t)Rc * Rc + (size_t)ranks[n] * Rc);
      TS_TRY(ensure_dynamic_smem((const void*)k_cp_update<T>, smem));
      k_cp_update<T><<<1, 256, smem, st>>>(d, n, Rc, fp, M, A[n], flag);
      TS_LAUNCH_CHECK();
    }
  }
  return TS_OK;
}

template <typename T>
ts_status launch_superdiag(int order, int Rc, T* D, cudaStream_t st) {
  long total = 1;
  for (int k = 0; k < order; ++k) total *= Rc;
  k_superdiag<T><<<grid_for(total), 256, 0, st>>>(order, Rc, D);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

#define TS_INST(T)                                                                           \
  template size_t cp_core_scratch_elems<T>(int, const int*, int);                           \
  template ts_status cp_als_core<T>(int, const int*, int, int, const T*, T* const*, T*, int*, \
                                    cudaStream_t);                                          \
  template ts_status launch_superdiag<T>(int, int, T*, cudaStream_t);
TS_INST(float)
TS_INST(double)
#undef TS_INST

}  // namespace ts

using namespace ts;

static bool cp_als_shape_ok(int32_t order, const int32_t* ranks, int32_t R_cp, int32_t dtype) {
  if (order < 2 || order > TS_MAX_ORDER || !ranks || R_cp < 1) return false;
  if (dtype != TS_F32 && dtype != TS_F64) return false;
  for (int k = 0; k < order; ++k)
    if (ranks[k] < 1 || R_cp > ranks[k]) return false;
  return true;
}

extern "C" size_t ts_cp_als_scratch_bytes(int32_t order, const int32_t* ranks, int32_t R_cp,
                                          int32_t dtype) {
  if (!cp_als_shape_ok(order, ranks, R_cp, dtype)) return 0;
  const size_t e = dtype == TS_F64 ? cp_core_scratch_elems<double>(order, ranks, R_cp) * 8
                                   : cp_core_scratch_elems<float>(order, ranks, R_cp) * 4;
  return 256 + e;
}

extern "C" ts_status ts_cp_als(int32_t order, const int32_t* ranks, int32_t R_cp, int32_t sweeps,
                               int32_t dtype, const void* core, void* const* factors_out,
                               void* scratch, size_t scratch_bytes, ts_stream stream) {
  clear_error();
  if (!cp_als_shape_ok(order, ranks, R_cp, dtype) || sweeps < 0)
    return fail(TS_ERR_SHAPE, "ts_cp_als: order %d, R_cp %d, sweeps %d (R_cp <= every rank)",
                order, R_cp, sweeps);
  if (!core || !factors_out || !scratch)
    return fail(TS_ERR_INVALID_ARG, "ts_cp_als: NULL argument");
  for (int k = 0; k < order; ++k)
    if (!factors_out[k]) return fail(TS_ERR_INVALID_ARG, "ts_cp_als: NULL factor %d", k);
  const size_t need = ts_cp_als_scratch_bytes(order, ranks, R_cp, dtype);
  if (scratch_bytes < need || (reinterpret_cast<uintptr_t>(scratch) & 255))
    return fail(TS_ERR_WORKSPACE, "ts_cp_als: need %zu bytes of 256-aligned scratch", need);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* flag = static_cast<int*>(scratch);
  TS_CUDA(cudaMemsetAsync(flag, 0, 256, st));
  char* rest = static_cast<char*>(scratch) + 256;
  if (dtype == TS_F64)
    return cp_als_core<double>(order, ranks, R_cp, sweeps, static_cast<const double*>(core),
                               reinterpret_cast<double* const*>(factors_out),
                               reinterpret_cast<double*>(rest), flag, st);
  return cp_als_core<float>(order, ranks, R_cp, sweeps, static_cast<const float*>(core),
                            reinterpret_cast<float* const*>(factors_out),
                            reinterpret_cast<float*>(rest), flag, st);
}
