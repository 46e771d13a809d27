// Internal launch interfaces shared by the translation units of libtsketch.
#pragma once

#include "common.cuh"

namespace ts {

// ---------------------------------------------------------------- hash.cu
ts_status launch_hash_table(uint64_t seed, int purpose, int sweep, int n, int k, int64_t size,
                            int nbins, int32_t* out, cudaStream_t st);
// out[e] = scale * N(0,1) draw e of the object (seed, tag), e in [0, count).
template <typename T>
ts_status launch_gaussian(uint64_t seed, uint64_t tag, int64_t count, double scale, T* out,
                          cudaStream_t st);

// ---------------------------------------------------------------- fft_ts.cu
constexpr int kMaxRadices = 32;
struct FftPlan {
  int m;
  int nst;
  int radix[kMaxRadices];
};
FftPlan make_fft_plan(int m);
template <typename T>
int fft_max_len();
template <typename T>
ts_status launch_twiddles(int m, Cx<T>* tw, cudaStream_t st);
// Z (column-major m x prod cols) = TensorSketch of factors[0] (x) ... (x) factors[nf-1].
// spectra: scratch of (sum cols) * m complex values; tw: twiddles from launch_twiddles.
template <typename T>
ts_status launch_ts_apply(int nf, const T* const* factors, const int64_t* rows, const int* cols,
                          const int32_t* const* tables, int m, const Cx<T>* tw, Cx<T>* spectra,
                          T* Z, cudaStream_t st);

// ---------------------------------------------------------------- input_sketch.cu
// One output of a pass over the data tensor: Y (nbins x dims[mode], row-major) =
// S T_(mode)^T with S the TensorSketch whose tables are tables[k], k != mode.
struct SketchJob {
  int mode;
  int nbins;
  void* out;
  const int32_t* tables[TS_MAX_ORDER];
};
constexpr int kMaxJobs = 2 * TS_MAX_ORDER;
// Zeroes every output, then accumulates all jobs in one pass over X.
template <typename T>
ts_status launch_input_sketch(const ts_tensor& X, const SketchJob* jobs, int njobs,
                              cudaStream_t st);

// ---------------------------------------------------------------- gemm.cu
// Strided matrix view: element (i, j) at p[i * rs + j * cs].
template <typename T>
struct MatView {
  const T* p;
  long rs, cs;
};
template <typename T>
struct OutView {
  T* p;
  long rs, cs;
};
// C = alpha * A B + beta * C for A (M x K), B (K x N).  `partial` (may be null)
// enables a deterministic split of K: up to partial_elems / (M N) slices.
template <typename T>
ts_status gemm(int M, int N, int K, double alpha, MatView<T> A, MatView<T> B, double beta,
               OutView<T> C, T* partial, size_t partial_elems, cudaStream_t st);

// ---------------------------------------------------------------- solve.cu
// Layout of the core for scattering C_(n)^T into it.
struct CoreMap {
  int order;
  int n;
  int ranks[TS_MAX_ORDER];
};

// RSVD-LRLS stage 1 (Alg. 5): with G = Z^T Z (r x r) and W = Z^T Y Omega (r x k):
// C = G^{-1} W, Q = orth(C) (FP64 Householder QR), E = G^{-1} Q.
template <typename T>
ts_status launch_rsvd_stage1(int r, int k, const T* G, const T* W, T* Q, T* E, int* flag,
                             cudaStream_t st);
// Shared memory of the stage-1 kernel; it must not exceed kMaxSmem.
inline size_t rsvd_stage1_smem_bytes(int r, int k, size_t tsize) {
  return sizeof(double) * (3 * (size_t)r * k + k + 2) + tsize * ((size_t)r * r + (size_t)r * k);
}
constexpr size_t kMaxSmem = 227 * 1024;
// X = G^{-1} H for G (r x r) SPD and H (r x s).
template <typename T>
ts_status launch_chol_solve(int r, int s, const T* G, const T* H, T* X, int* flag,
                            cudaStream_t st);
// Symmetric eigen-decomposition of K (n x n), eigenvalues descending, lambda_i = sigma_i^2:
// CnT = Q U_R Sigma_R (r x R; Q null means identity, r = n), Fm = U_R Sigma_R^{-1} (n x R),
// Uout = U_R (n x R).  Any output may be null.
template <typename T>
ts_status launch_eig_small(int n, int R, const T* K, const T* Q, int r, T* CnT, T* Fm, T* Uout,
                           int* flag, cudaStream_t st);
constexpr int kMaxEig = 64;
constexpr int kMaxCholSmem = 192;
// Column signs (largest-|.| entry positive) on V (s x R); flips CnT (r x R) with it,
// writes A_out = V and, when core != null, scatters CnT into the core.
template <typename T>
ts_status launch_finalize(int s, int R, const T* V, T* A_out, T* CnT, int r, T* core,
                          CoreMap map, cudaStream_t st);

// ---------------------------------------------------------------- leverage.cu
// Leverage-score sketch of subproblem `mode` (dense X).  Z column-major m x prod R_k,
// Y m x dims[mode]; samples m x (order-1); scratch: leverage_scratch_doubles() doubles.
size_t leverage_scratch_doubles(const ts_tensor& X, int mode, int m);
template <typename T>
ts_status launch_leverage(const ts_tensor& X, int mode, const int* ranks, const T* const* factors,
                          int m, uint64_t seed, int sweep, T* Z, T* Y, int32_t* samples,
                          double* scratch, cudaStream_t st);

// ---------------------------------------------------------------- cp.cu
// HOSVD initialisation and CP-ALS sweeps on a core of the given ranks; A[k] is
// ranks[k] x Rc.  scratch: cp_core_scratch_elems<T>() values.
template <typename T>
size_t cp_core_scratch_elems(int order, const int* ranks, int Rc);
template <typename T>
ts_status cp_als_core(int order, const int* ranks, int Rc, int sweeps, const T* core, T* const* A,
                      T* scratch, int* flag, cudaStream_t st);
// D (Rc^order, C order) = superdiagonal tensor of ones.
template <typename T>
ts_status launch_superdiag(int order, int Rc, T* D, cudaStream_t st);

// ---------------------------------------------------------------- fit.cu
template <typename T>
size_t fit_dense_scratch_elems(const ts_tensor& X, const int* ranks);
template <typename T>
ts_status launch_fit_dense(const ts_tensor& X, const int* ranks, const T* core,
                           const T* const* factors, T* scratch, double* acc, double* residual_out,
                           cudaStream_t st);

}  // namespace ts
