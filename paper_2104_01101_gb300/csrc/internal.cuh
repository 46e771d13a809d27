// Internal launch interfaces shared by the translation units of libtsketch.
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace ts {

// cuTensorMapEncodeTiled, obtained from the driver once (TMA tensor maps).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
ts_status encode_fn(EncodeTiledFn* out);

// ---------------------------------------------------------------- hash.cu
ts_status launch_hash_table(uint64_t seed, int purpose, int sweep, int n, int k, int64_t size,
                            int nbins, int32_t* out, cudaStream_t st);
// out[e] = scale * N(0,1) draw e of the object (seed, tag), e in [0, count).
template <typename T>
ts_status launch_gaussian(uint64_t seed, uint64_t tag, int64_t count, double scale, T* out,
                          cudaStream_t st);
// Gaussian test matrices of Alg. 5 for sweeps sweep0 .. sweep0 + nsweeps - 1 of every mode
// in one launch.  Mode n's block (rows[n] x nsweeps k[n], row-major) starts at off[n];
// blocks are contiguous in mode order and total = off[N-1] + rows[N-1] nsweeps k[N-1].
// Columns [t k[n], (t+1) k[n]) hold Omega(sweep0 + t, n).
struct OmegaBlocks {
  int N, nsweeps, sweep0;
  int64_t rows[TS_MAX_ORDER];
  int k[TS_MAX_ORDER];
  int64_t off[TS_MAX_ORDER];
  int64_t total;
};
template <typename T>
ts_status launch_omegas(uint64_t seed, const OmegaBlocks& ob, T* out, cudaStream_t st);

// ---------------------------------------------------------------- fft_ts.cu
constexpr int kMaxRadices = 32;
struct FftPlan {
  int m;
  int nst;
  int stage_tw;  // 1: kernels copy the twiddle table into shared memory first
  int radix[kMaxRadices];
};
FftPlan make_fft_plan(int m);
template <typename T>
int fft_max_len();
template <typename T>
ts_status launch_twiddles(int m, Cx<T>* tw, cudaStream_t st);
// The factor chain of one TensorSketch: factors, their rows and columns, their tables.
struct ChainDesc {
  int nf;
  int total_cols;
  const void* factors[TS_MAX_ORDER];
  int64_t rows[TS_MAX_ORDER];
  int cols[TS_MAX_ORDER];
  int colbase[TS_MAX_ORDER];
  const int32_t* tables[TS_MAX_ORDER];
};
// One TensorSketch of a batch: chain, FFT plan, twiddles, spectra scratch, output Z.
template <typename T>
struct TsChainJob {
  ChainDesc d;
  FftPlan plan;
  int ncols;  // prod cols: the columns of Z
  const Cx<T>* tw;
  Cx<T>* spectra;
  T* Z;
};
template <typename T>
TsChainJob<T> make_chain_job(int nf, const T* const* factors, const int64_t* rows,
                             const int* cols, const int32_t* const* tables, int m,
                             const Cx<T>* tw, Cx<T>* spectra, T* Z);
template <typename T>
size_t chain_job_smem(const TsChainJob<T>& j);
// jobs: device array of count chain jobs; the grids are max_spectra_blocks (ceil of the
// largest total_cols / 2) and max_z_blocks (ceil of the largest ncols / 2) by count;
// smem: the largest chain_job_smem.
template <typename T>
ts_status launch_ts_apply_batched(const TsChainJob<T>* jobs, int count, int max_spectra_blocks,
                                  int max_z_blocks, size_t smem, cudaStream_t st);
// Adjoint of launch_ts_apply: given dZ = dL/dZ (column-major m x prod cols) and the
// factor spectra the forward call left in `spectra`, writes dL/d(factor f) into
// grads[f] (HOST array of nf device pointers, rows[f] x cols[f] row-major).
// dspec: m x prod cols complex scratch; dU: m x (sum cols) real scratch.
template <typename T>
ts_status launch_ts_adjoint(int nf, const int64_t* rows, const int* cols,
                            const int32_t* const* tables, int m, const Cx<T>* tw,
                            const Cx<T>* spectra, const T* dZ, Cx<T>* dspec, T* dU,
                            T* const* grads, cudaStream_t st);
// Z (column-major m x prod cols) = TensorSketch of factors[0] (x) ... (x) factors[nf-1].
// spectra: scratch of (sum cols) * m complex values; tw: twiddles from launch_twiddles.
// Zb_bf16 (FP32 only, nullable): Z^T also written in BF16, row c of Z^T at c * ldb.
template <typename T>
ts_status launch_ts_apply(int nf, const T* const* factors, const int64_t* rows, const int* cols,
                          const int32_t* const* tables, int m, const Cx<T>* tw, Cx<T>* spectra,
                          T* Z, cudaStream_t st, void* Zb_bf16 = nullptr, int ldb = 0);

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
// Zeroes every output, then accumulates all jobs in one pass over X.  Dense order-3
// FP32 tensors with at most one job per mode take the TMA tile/bulk-reduction kernel
// (input_sketch_tma.cu); a bounded wait that expires there writes TS_ERR_TIMEOUT to
// *flag (when flag is not null).
template <typename T>
ts_status launch_input_sketch(const ts_tensor& X, const SketchJob* jobs, int njobs, int* flag,
                              cudaStream_t st);
bool dense3_tma_eligible(const ts_tensor& X, const SketchJob* jobs, int njobs);
size_t dense3_tma_smem_bytes(const ts_tensor& X, const SketchJob* jobs, int njobs);
ts_status launch_dense3_tma(const ts_tensor& X, const SketchJob* jobs, int njobs, int* flag,
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
// C = alpha * A B + beta * C for A (M x K), B (K x N).  With a GemmSplit the long
// dimension K may be split across CTAs; the partials are then summed in split order
// by a second kernel (deterministic).
template <typename T>
struct GemmSplit {
  T* partial;            // splits x M x N values
  size_t partial_elems;
  unsigned* counters;    // unused (kept for layout stability of the workspaces)
  int ncounters;
  const int* skip;       // nullable device flag: non-zero when the product's kernels start
                         // (after the previous kernel completed) makes them return at once
};
template <typename T>
ts_status gemm(int M, int N, int K, double alpha, MatView<T> A, MatView<T> B, double beta,
               OutView<T> C, const GemmSplit<T>* split, cudaStream_t st);
// Same, with B's columns [0, n1) taken from B1 and [n1, N) from B2 (column j - n1).
template <typename T>
ts_status gemm2(int M, int N, int K, double alpha, MatView<T> A, MatView<T> B1, int n1,
                MatView<T> B2, double beta, OutView<T> C, const GemmSplit<T>* split,
                cudaStream_t st);
// Same, with B's columns [0, n1) from B1, [n1, n2) from B2 (column j - n1) and [n2, N)
// from B3 (column j - n2).
template <typename T>
ts_status gemm3(int M, int N, int K, double alpha, MatView<T> A, MatView<T> B1, int n1,
                MatView<T> B2, int n2, MatView<T> B3, double beta, OutView<T> C,
                const GemmSplit<T>* split, cudaStream_t st);
constexpr int kGemmCounters = 4096;
// tall_products.cu: products with a huge dimension s (used from kTallMinS on).
constexpr long kTallMinS = 16384;
// D (k x s, row stride ldd) = M^T Y, M (m x k, row stride ldm, k <= 32), Y (m x s, ldy);
// the rows may be split over blocks, their partials (in `part`) summed in order.
template <typename T>
ts_status tall_tn(int m, int k, long s, const T* M, long ldm, const T* Y, long ldy, T* D,
                  long ldd, T* part, size_t part_elems, cudaStream_t st);
// K (k x k, row stride ldk) = D D^T, D (k x s, row stride ldd), k <= 32; through `part`
// (min(304, ceil(s / 1024)) k^2 values).
template <typename T>
ts_status gram_wide(int k, long s, const T* D, long ldd, T* K, long ldk, T* part,
                    size_t part_elems, cudaStream_t st);
// P (m x n; element (i, c) at P[i prs + c pcs]) = Y (m x s, ldy) Om (s x n, ldo), summed
// over chunks of s through `part` (chunks x m x min(n, 80) values).
template <typename T>
ts_status wide_nn(int m, int n, long s, const T* Y, long ldy, const T* Om, long ldo, T* P,
                  long prs, long pcs, T* part, size_t part_elems, cudaStream_t st);
// One product of a batch: C (M x N) = A (M x K) [B1 | B2 | B3] (columns [0, n1) of B from
// B1, [n1, n2) from B2, [n2, N) from B3).
template <typename T>
struct GemmJob {
  int M, N, K, n1, n2;
  MatView<T> A, B1, B2, B3;
  OutView<T> C;
};
// jobs: device array of count products; grid from the largest M and N; tile 32 or 64.
template <typename T>
ts_status launch_gemm_batched(const GemmJob<T>* jobs, int count, int maxM, int maxN, int tile,
                              cudaStream_t st);
// C (M x N, row stride ldc) = sum over splits of partial (split-major M x N).
template <typename T>
ts_status launch_split_reduce(int M, int N, int splits, const T* partial, T* C, long ldc,
                              cudaStream_t st);

// ---------------------------------------------------------------- gram_tc.cu
// BF16 precision form of the Gram products (tcgen05): operands are BF16 row-major with
// a row stride of gram_tc_ld(K) elements (16-byte rows).  pack_bf16 writes rows x K of
// src (element (i, k) at src[i rs + k cs]); gram_tc_map encodes a TMA map over such a
// buffer; gram_tc forms C (M x N, row stride ldc) = A B^T, summing split-K partials
// (gram_tc_partial_elems floats) in split order.
int gram_tc_ld(int K);
ts_status pack_bf16(const float* src, long rs, long cs, int rows, int K, void* dst,
                    cudaStream_t st);
ts_status gram_tc_map(const void* base, int rows, int K, CUtensorMap* map);
size_t gram_tc_partial_elems(int M, int N, int K);
ts_status gram_tc(const CUtensorMap& mapA, const CUtensorMap& mapB, int M, int N, int K,
                  float* C, long ldc, float* partial, int* flag, cudaStream_t st);

// ---------------------------------------------------------------- solve.cu
// Layout of the core for scattering C_(n)^T into it.
struct CoreMap {
  int order;
  int n;
  int ranks[TS_MAX_ORDER];
};

constexpr size_t kMaxSmem = 227 * 1024;
constexpr int kMaxEig = 64;
// RSVD-LRLS stage 1 (Alg. 5): with G = Z^T Z (r x r, row stride ldg) and
// W = Z^T Y Omega (r x k, row stride ldw): C = G^{-1} W, Q = orth(C) (Householder,
// FP64 when qr64), E = G^{-1} Q.
template <typename T>
ts_status launch_rsvd_stage1(int r, int k, const T* G, int ldg, const T* W, int ldw, T* Q, T* E,
                             bool qr64, int* flag, cudaStream_t st);
size_t rsvd_stage1_smem_bytes(int r, int k, size_t tsize, bool qr64);
// Large-r pieces of stage 1: Q = orth(C) in one block, and G^{-1} by Newton-Schulz
// (S1: 2 r^2 values, S2: r^2 values of scratch; conv: 3 device ints, or null, through
// which the steps after convergence return at once).
template <typename T>
ts_status launch_qr_only(int r, int k, const T* C, T* Q, bool qr64, cudaStream_t st);
size_t qr_only_smem_bytes(int r, int k, bool qr64, size_t tsize);
template <typename T>
ts_status newton_schulz_inverse(int r, const T* G, long ldg, T* X, T* S1, T* S2, int iters,
                                int* conv, const GemmSplit<T>* split, cudaStream_t st);
constexpr int kNewtonSchulzIters = 14;
// X = G^{-1} H for G (r x r) SPD and H (r x s).
template <typename T>
ts_status launch_chol_solve(int r, int s, const T* G, const T* H, T* X, int* flag,
                            cudaStream_t st);
size_t chol_solve_smem_bytes(int r, size_t tsize);
// Symmetric eigen-decomposition of K (n x n), eigenvalues descending, lambda_i = sigma_i^2:
// CnT = Q U_R Sigma_R (r x R; Q null means identity, r = n), Fm = U_R Sigma_R^{-1} (n x R),
// Uout = U_R (n x R).  Any output may be null.  polish64: FP64 final sweeps (FP32 data).
template <typename T>
ts_status launch_eig_small(int n, int R, const T* K, const T* Q, int r, T* CnT, T* Fm, T* Uout,
                           bool polish64, int* flag, cudaStream_t st);
// The whole subproblem in one block (lrls_fused.cu) after [G | W | H] =
// Z^T [Z | Y Omega | Y] (RSVD) or [G | H] = Z^T [Z | Y] (exact, W unused): writes A_out
// (s x R), CnT (r x R, may be null) and the core (may be null).  Mbuf: k x s scratch,
// used when D does not fit on chip.  lrls_fused_supported() tells whether the shape fits.
size_t lrls_fused_smem_bytes(int r, int s, int k, int R, int solve, size_t tsize, bool fp64,
                             bool* m_smem);
bool lrls_fused_supported(int r, int s, int k, int R, int solve, size_t tsize, bool fp64);
// Arguments of the single-block solve of one subproblem (see launch_lrls_fused).
template <typename T>
struct FusedArgs {
  int r, s, k, R, solve;
  const T* G;
  long ldg;  // r x r
  const T* W;
  long ldw;  // r x k (RSVD)
  const T* H;
  long ldh;   // r x s
  T* Mbuf;    // k x s when D is not kept on chip
  T* CnT;     // r x R out (may be null)
  T* A_out;   // s x R out
  T* core;    // may be null
  CoreMap map;
  int* flag;
  bool m_smem;
};
// The arguments and dynamic shared memory of one subproblem; TS_ERR_SHAPE when it does
// not fit one block.
template <typename T>
ts_status make_fused_args(int r, int s, int k, int R, int solve, bool fp64, const T* G, long ldg,
                          const T* W, long ldw, const T* H, long ldh, T* Mbuf, T* CnT, T* A_out,
                          T* core, CoreMap map, int* flag, FusedArgs<T>* out, size_t* smem);
// count subproblems (device array of arguments), one block each; smem: the largest.
template <typename T>
ts_status launch_lrls_fused_batched(const FusedArgs<T>* args, int count, bool fp64, size_t smem,
                                    cudaStream_t st);
template <typename T>
ts_status launch_lrls_fused(int r, int s, int k, int R, int solve, bool fp64, const T* G,
                            long ldg, const T* W, long ldw, const T* H, long ldh, T* Mbuf, T* CnT,
                            T* A_out, T* core, CoreMap map, int* flag, cudaStream_t st);
// lrls_chol.cu: the RSVD subproblem by symmetric elimination of [G | W] in registers
// (r + k <= 128, k <= 16); the same arguments as the fused solve (m_smem is recomputed);
// fp64 (FP32 data): the precision form, the QR of C and K's eigen-decomposition in FP64.
bool lrls_chol_supported(int r, int s, int k, int R, int solve, size_t tsize, bool fp64);
template <typename T>
ts_status launch_lrls_chol(const FusedArgs<T>& a, bool fp64, cudaStream_t st);
// lrls_chol.cu: the symmetric eigensolver for n <= 16 (Jacobi on four warps; fp64 with
// FP32 data: one FP64 refinement), with the outputs of launch_eig_small.
template <typename T>
ts_status launch_eig16(int n, int R, const T* K, const T* Q, int r, T* CnT, T* Fm, T* Uout,
                       bool fp64, int* flag, cudaStream_t st);
// Factor columns V (s x R) with V(i, c) = sum_a M(i, a) Fm(a, c) (M element (i, a) at
// M[i*rs + a*cs], a < kdim), or V(i, c) = M[i*rs + c*cs] when Fm is null.  Each
// column is signed so that its largest-|.| entry is positive; A_out = V; CnT (r x R)
// is flipped with it and, when core != null, scattered into the core.  Tall columns
// (s >= 6145) run over many blocks when `scratch` (stream-ordered, free) holds the
// chunk maxima: nb * R * (sizeof(T) + 4) + 256 bytes, nb = ceil(s / max(2048, ceil(s / 256))).
template <typename T>
ts_status launch_finalize(int s, int R, const T* M, long rs, long cs, int kdim, const T* Fm,
                          T* A_out, T* CnT, int r, T* core, CoreMap map, cudaStream_t st,
                          void* scratch = nullptr, size_t scratch_bytes = 0);

// ---------------------------------------------------------------- fibre_index.cu
// Hash index of the mode-`mode` fibres of a COO tensor (device arrays; passed to
// kernels by value).  Slot h of the table (capacity mask + 1) holds key keys[h] (the
// C-order linear index of the other coordinates, ~0 when empty) and owns the entries
// beg[h] .. beg[h+1]-1 of pos (mode-`mode` coordinate) and val (value, X's dtype).
struct FibreIndex {
  int order, mode;
  int64_t stride[TS_MAX_ORDER];  // key = sum_{k != mode} i_k stride[k]
  uint64_t mask;
  unsigned long long* keys;
  int32_t* beg;   // capacity + 1
  int32_t* cur;   // capacity (counts, then fill cursors)
  int32_t* pos;   // nnz
  void* val;      // nnz
  int32_t* part;  // scan partials
};
int64_t fibre_index_capacity(int64_t nnz);
bool fibre_keys_fit(const ts_tensor& X, int mode);
// Carves one mode's index from b (sizes from X.nnz and X.dtype).
FibreIndex fibre_index_carve(const ts_tensor& X, int mode, Bump& b);
// Builds it from the COO tensor X; sets *flag = 2 if a key finds no slot (excluded by
// the capacity >= 2 nnz).
ts_status launch_fibre_index_build(const ts_tensor& X, const FibreIndex& F, int* flag,
                                   cudaStream_t st);
// The keys only (no counts, ranges or entries): eslot[e] = the slot of nonzero e's fibre.
ts_status launch_fibre_keys(const ts_tensor& X, const FibreIndex& F, int32_t* eslot, int* flag,
                            cudaStream_t st);

// ---------------------------------------------------------------- fit_coo.cu
// Residual of a Tucker model against a COO tensor.  Scratch: the fibre index of the
// largest mode, a hash table merging repeated coordinates, the Gram matrices
// G_n = A^(n)T A^(n) (stride gstride elements), two core-sized buffers and
// acc[4] (acc[1] = <T, T~>, acc[2] = ||T~||^2, acc[3] = ||T||^2).
struct FitCooWork {
  FibreIndex F;       // keys of the largest mode's fibres (no ranges or entries)
  int32_t* eslot;     // nnz: fibre slot of every nonzero
  unsigned long long* vkeys;
  double* vsum;
  uint64_t vmask;
  void* G;
  int gstride;
  void* M1;
  void* M2;
  double* acc;
};
bool fit_coo_supported(const ts_tensor& X);  // order >= 2, < 2^30 nonzeros, keys fit
bool fit_coo_model_ok(const ts_tensor& X, const int* ranks);  // core <= 200 KB, last rank <= 64
FitCooWork fit_coo_carve(const ts_tensor& X, const int* ranks, Bump& b);
// ||T||^2 with repeated coordinates merged, into acc[3] (once per tensor).
ts_status launch_fit_coo_norm(const ts_tensor& X, const FitCooWork& w, int* flag,
                              cudaStream_t st);
// The relative residual into *residual (after launch_fit_coo_norm on the same work).
template <typename T>
ts_status launch_fit_coo(const ts_tensor& X, const int* ranks, const T* core,
                         const T* const* factors, const FitCooWork& w, double* residual,
                         cudaStream_t st);

// ---------------------------------------------------------------- leverage.cu
// Leverage-score sketch of subproblem `mode`.  Z column-major m x prod R_k,
// Y m x dims[mode]; samples m x (order-1); scratch: leverage_scratch_doubles() doubles.
// A COO tensor needs `fib`, the built fibre index of `mode`.
// The deterministic selection scores every one of the C = prod_{k != mode} dims[k]
// candidate rows; it runs when C <= kLevDetMaxCandidates.
constexpr int64_t kLevDetMaxCandidates = int64_t(1) << 31;
int64_t leverage_det_candidates(const ts_tensor& X, int mode);  // C, or -1 above the limit
size_t leverage_scratch_doubles(const ts_tensor& X, int mode, int m);
template <typename T>
ts_status launch_leverage(const ts_tensor& X, int mode, const int* ranks, const T* const* factors,
                          int m, uint64_t seed, int sweep, T* Z, T* Y, int32_t* samples,
                          double* scratch, cudaStream_t st,
                          bool det = false, const FibreIndex* fib = nullptr);

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
