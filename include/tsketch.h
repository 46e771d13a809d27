/*
 * tsketch.h -- C ABI of the GB300 sketched Tucker-ALS library (libtsketch.so).
 *
 * Method: Ma & Solomonik, "Fast and accurate randomized algorithms for low-rank
 * tensor decompositions" (arXiv 2104.01101).  The library computes the hot path
 * of Sketch-Tucker-ALS (Alg. 4): TensorSketch of the factor Kronecker chain by
 * CountSketch -> FFT -> Hadamard -> inverse FFT (Sec. 3.1), the one-pass sketch
 * of the data tensor's unfoldings (Alg. 4, right-hand side), leverage-score
 * sampling (Sec. 3.2), the randomized range finder initialisation (Alg. 3 with
 * the composite sketch of Sec. 5), the sketched rank-constrained solve
 * (RSVD-LRLS, Alg. 5, or the exact truncated solve of Theorem 4.1) and the
 * fitness of Sec. 7; plus CP-ALS on the Tucker core (Alg. 6).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Memory: every array argument is a DEVICE pointer owned by the caller unless
 *   the comment says "host".  The library never allocates device memory: calls
 *   that need scratch take (scratch, scratch_bytes) and publish the size they
 *   need through a *_bytes query.  Scratch must be 256-byte aligned.
 * - Streams: all work is enqueued on `stream` (a cudaStream_t; NULL = legacy
 *   default stream) and is asynchronous unless stated otherwise.  The returned
 *   status covers argument validation and launch errors only; faults inside a
 *   kernel surface at the caller's next synchronisation.
 * - Errors: on any status other than TS_OK, ts_last_error() returns a message
 *   for the calling thread.  Nothing is written to outputs on validation errors.
 * - Layouts: matrices are row-major; a "s x R factor" is s rows of R contiguous
 *   values.  Dense tensors are C order (last mode fastest).  Unfoldings,
 *   Kronecker chains and the core follow C order: column (r_k)_{k != n} of
 *   P^(n) = A^(1) (x) ... (x) A^(N) (mode n skipped) has the lowest mode slowest.
 * - Hash tables: int32 per index, bucket in bits 0..30 and bit 31 set when the
 *   sign is -1 (see ts_hash_table).
 * - Modes are 0-based (the paper's mode n is mode n-1 here).
 */
#ifndef TSKETCH_H
#define TSKETCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* ts_stream; /* == cudaStream_t */

typedef enum {
  TS_OK = 0,
  TS_ERR_INVALID_ARG = 1, /* null pointer, bad enum, negative size */
  TS_ERR_SHAPE = 2,       /* sizes violate the method's assumptions (see each call) */
  TS_ERR_WORKSPACE = 3,   /* scratch too small or misaligned */
  TS_ERR_CUDA = 4,        /* a CUDA runtime call failed */
  TS_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  TS_ERR_NUMERIC = 6,     /* non-finite value or non-positive-definite Gram */
  TS_ERR_UNSUPPORTED = 7  /* valid request outside what this build implements */
} ts_status;

typedef enum { TS_F32 = 0, TS_F64 = 1 } ts_dtype;
typedef enum { TS_DENSE = 0, TS_COO = 1 } ts_format;
typedef enum { TS_TENSORSKETCH = 0, TS_LEVERAGE = 1, TS_LEVERAGE_DET = 2 } ts_sketch_kind;
typedef enum { TS_SOLVE_RSVD = 0, TS_SOLVE_EXACT = 1 } ts_solve_kind;

/* Purposes of the library's random objects (the top byte of their tag). */
enum {
  TS_PURPOSE_TS_HASH = 1,     /* TensorSketch bucket/sign maps H_{n,k}, S_{n,k} */
  TS_PURPOSE_RRF_HASH = 2,    /* CountSketch factor of the composite sketch */
  TS_PURPOSE_RRF_GAUSS = 3,   /* Gaussian factor of the composite sketch */
  TS_PURPOSE_RSVD_GAUSS = 4,  /* Gaussian test matrix of RSVD-LRLS */
  TS_PURPOSE_LEV_UNIFORM = 5  /* uniforms of leverage-score sampling */
};

#define TS_MAX_ORDER 8

/* An order-N tensor held on the device.
 * format TS_DENSE: `values` holds prod(dims) elements in C order.
 * format TS_COO:   `indices` holds N arrays of nnz int32 coordinates, mode after
 *                  mode (structure of arrays: indices[k*nnz + e]); `values` holds
 *                  nnz values.  Repeated coordinates add (every operation here is
 *                  linear in the entries).  Coordinates must lie in [0, dims[k]): the
 *                  kernels skip entries outside rather than read out of bounds, and
 *                  results for such input are unspecified.
 * dtype: element type of `values` (TS_F32 or TS_F64). */
typedef struct {
  int32_t order;
  int64_t dims[TS_MAX_ORDER];
  int32_t format;
  int32_t dtype;
  const void* values;
  const int32_t* indices;
  int64_t nnz;
} ts_tensor;

/* Options of tucker_als_sketched / cp_via_tucker.  Zero-initialise, then set. */
typedef struct {
  uint64_t seed;              /* names every random object (hash tables, Gaussians, uniforms) */
  int32_t rrf_k1;             /* composite-sketch width k1 (Alg. 3); 0 = ceil(sqrt(m)) */
  int32_t rrf_k2;             /* CountSketch width k2; 0 = R^2 + k1 */
  int32_t rsvd_oversample;    /* p in the k = R + p columns of Alg. 5's test matrix; <0 = 5 */
  int32_t solve;              /* ts_solve_kind; TS_SOLVE_RSVD is the routine Alg. 4 calls */
  int32_t resketch_each_sweep;/* 1: redraw TensorSketch tables and re-sketch T every sweep */
  int32_t gram_bf16;          /* 1 (FP32 data): the product [Z^T Z | Z^T Y Omega | Z^T Y]
                                 of every subproblem solved in one block runs in BF16 on
                                 the tensor cores with FP32 accumulation (the precision
                                 form); the sketches and the solve stay FP32 */
  int32_t init_given;         /* 1: factors_inout already hold the initial A^(2..N) (no RRF) */
  int32_t track_fit;          /* 1: write the relative residual after every sweep */
  int32_t solve_fp64;         /* FP32 data: 1 runs the QR of Alg. 5 and the SVD's
                                 eigenpairs in FP64 (slower on GB300): in the cluster solve
                                 (r + k <= 128, k <= 16) FP64 CholeskyQR2 and one FP64
                                 refinement of the FP32 Jacobi's eigenpairs, in the other
                                 solves an FP64 Householder QR and an FP64 polish of the
                                 eigenpairs; FP64 data always solves in FP64 */
  int32_t use_graph;          /* 1: capture the whole decomposition as a CUDA graph on first
                                 use (cached per argument set and device, up to 8 entries) and
                                 replay it on later calls with identical arguments.  The
                                 first call pays for the capture; it must not itself be made
                                 while the caller's thread is capturing a stream. */
  /* Optional profiling hook: HOST array of 6 cudaEvent_t (or NULL).  The driver
   * records them on `stream` at: [0] call start, [1] after Init-RRF, [2] before
   * the one-pass sketch of the data tensor, [3] after it, [4] after the last
   * sweep, [5] after the residual.  Ignored when use_graph is set. */
  void* const* phase_events;
} ts_options;

/* Message describing the last error on the calling thread ("" if none). */
const char* ts_last_error(void);

/* Library version string (static storage). */
const char* ts_version(void);

/* Number of CUDA kernels this library has launched in the calling process
 * (a monotone counter, for profiling). */
uint64_t ts_kernel_launches(void);

/* ------------------------------------------------------------------------- */
/* Hash tables (Sec. 3.1, TensorSketch definition; Sec. 5 composite sketch).
 *
 * Writes table_out[i], i in [0, size), for the random map named by
 * (seed, purpose, sweep, n, k): bucket = poly2(i) mod nbins and sign = +1 if
 * poly3(i) is even, else -1, where poly2/poly3 are polynomials of degree 2 and 3
 * over Z_p, p = 2^31 - 1, whose coefficients are splitmix64 outputs reduced mod p
 * (a 3-wise independent bucket map and a 4-wise independent sign map, as the
 * TensorSketch definition requires).  Integer-only: bit-identical to the oracle.
 * Errors: TS_ERR_INVALID_ARG if size < 0, size >= 2^31-1, nbins < 1, purpose,
 * n or k outside [0,256), sweep outside [0, 2^24), or table_out == NULL. */
ts_status ts_hash_table(uint64_t seed, int32_t purpose, int32_t sweep, int32_t n, int32_t k,
                        int64_t size, int32_t nbins, int32_t* table_out, ts_stream stream);

/* ------------------------------------------------------------------------- */
/* TensorSketch of a Kronecker chain (Sec. 3.1, FFT identity for SP).
 *
 * Computes Z = S P with P = F_0 (x) F_1 (x) ... (x) F_{nf-1} (F_j has rows[j] x
 * cols[j] entries, row-major) and S the TensorSketch whose per-factor tables are
 * tables[j] (rows[j] packed entries, buckets < m).  Each factor is CountSketched
 * to m x cols[j], transformed by an FFT of length m, the spectra are multiplied
 * over every column multi-index (factor 0 slowest) and inverse transformed.
 * Z_out: m x prod(cols) stored COLUMN-major (column c occupies Z_out[c*m .. c*m+m)).
 * factors, rows, cols, tables are HOST arrays of nf entries (the factor and
 * table pointers they hold are device pointers).
 * dtype: TS_F32 (FFT in FP32) or TS_F64.
 * Errors: TS_ERR_SHAPE if nf < 1 or > TS_MAX_ORDER-1, m < 2, or m too long for
 * the shared-memory FFT (m > 12288 in FP32, m > 6144 in FP64);
 * TS_ERR_WORKSPACE if scratch_bytes < tensorsketch_apply_scratch_bytes(). */
size_t tensorsketch_apply_scratch_bytes(int32_t nf, const int32_t* cols, int32_t m, int32_t dtype);
ts_status tensorsketch_apply(int32_t nf, const void* const* factors, const int64_t* rows,
                             const int32_t* cols, const int32_t* const* tables, int32_t m,
                             int32_t dtype, void* Z_out, void* scratch, size_t scratch_bytes,
                             ts_stream stream);

/* TensorSketch of a Kronecker chain WITHOUT caller scratch (no counterpart in the
 * paper: this is a library convenience).
 *
 * Same operation, arguments and errors as tensorsketch_apply, but the scratch
 * (twiddle table and factor spectra) lives in a fixed 8 MiB device array inside
 * the library, so the call allocates nothing: it makes no cudaMalloc/cudaFree
 * call and uses no allocating library routine.  It is meant for callers that
 * cannot allocate device memory at the point of the call: a plug-in running
 * inside a host application whose framework owns all device memory and hands it
 * no allocator, or a latency-critical path where cudaMalloc's implicit device
 * synchronisation is not acceptable.
 * - Limit: problems needing more than tensorsketch_apply_static_scratch_capacity()
 *   bytes (tensorsketch_apply_scratch_bytes) return TS_ERR_WORKSPACE.
 * - Cost: every GPU that loads the library holds the 8 MiB array until the process
 *   exits.
 * - Set-up: the first call on each device looks up the array's device address
 *   with that device current (cudaGetSymbolAddress) and caches it; make that first
 *   call before any stream capture.  The cache assumes the device's primary context
 *   lives until the process exits: after cudaDeviceReset the library's module is
 *   loaded again and the cached address may be stale, so do not call this entry
 *   point after resetting a device that it has already been called on.
 * - Concurrency: all calls share the one array and it keeps the last call's
 *   contents; calls that overlap on the GPU (any streams, any host threads) race,
 *   so order them (one stream, or events).  Nothing in it needs clearing: each
 *   call writes every scratch element it reads. */
size_t tensorsketch_apply_static_scratch_capacity(void);
ts_status tensorsketch_apply_static_scratch(int32_t nf, const void* const* factors,
                                            const int64_t* rows, const int32_t* cols,
                                            const int32_t* const* tables, int32_t m,
                                            int32_t dtype, void* Z_out, ts_stream stream);

/* ------------------------------------------------------------------------- */
/* One-pass sketch of the data tensor (Alg. 4, right-hand side Y = S^(n) T_(n)^T).
 *
 * For every stored entry (i, v) of X: Y[(sum_{k != mode} H_k(i_k)) mod m, i_mode]
 * += prod_{k != mode} S_k(i_k) * v.  tables is a HOST array of X->order device
 * pointers; tables[k] has dims[k] packed entries; tables[mode] is ignored.
 * Y_out: m x dims[mode] row-major in X's dtype, overwritten.
 * Errors: TS_ERR_SHAPE if order < 2 or > TS_MAX_ORDER or mode out of range. */
ts_status tensorsketch_input(const ts_tensor* X, int32_t mode, const int32_t* const* tables,
                             int32_t m, void* Y_out, ts_stream stream);

/* ------------------------------------------------------------------------- */
/* The Gram products of Alg. 5 in the BF16 precision form (the tensor-core path of the
 * sketched solve): C = bf16(A) bf16(B)^T accumulated in FP32.  A (M x K) and B (N x K)
 * are FP32 row-major device arrays, C (M x N) FP32 row-major; in the decomposition
 * A = Z^T and B = [Z | Y Omega | Y]^T.  The operands are rounded to BF16 (nearest, ties
 * to even) in scratch; each product of two BF16 values is exact in FP32, so C differs
 * from the exact product of the rounded operands only by the FP32 accumulation.  K is
 * split across CTAs and the partial sums are added in split order (deterministic).
 * Errors: TS_ERR_SHAPE unless M, N, K >= 1; TS_ERR_WORKSPACE for short or misaligned
 * scratch. */
size_t ts_gram_bf16_scratch_bytes(int32_t M, int32_t N, int32_t K);
ts_status ts_gram_bf16(int32_t M, int32_t N, int32_t K, const void* A, const void* B,
                       void* C_out, void* scratch, size_t scratch_bytes, ts_stream stream);

/* ------------------------------------------------------------------------- */
/* Init-RRF for one mode (Alg. 3 with the composite sketch of Sec. 5).
 *
 * B = T_(mode) S with S = T G: T a CountSketch of the prod_{k != mode} dims[k]
 * columns into k2 buckets (hashed with the restricted TensorSketch form of Sec.
 * 3.1, tables of purpose TS_PURPOSE_RRF_HASH), G a k2 x k1 Gaussian with
 * variance 1/k1.  A_out (dims[mode] x R, X's dtype) = the R leading left
 * singular vectors of B, each column signed so that its largest-magnitude entry
 * is positive.
 * Errors: TS_ERR_SHAPE unless 1 <= R <= k1 <= min(k2, dims[mode]) and
 * k2 <= prod_{k != mode} dims[k], or k1 > 64. */
size_t range_finder_init_scratch_bytes(const ts_tensor* X, int32_t mode, int32_t R, int32_t k1,
                                       int32_t k2);
ts_status range_finder_init(const ts_tensor* X, int32_t mode, int32_t R, int32_t k1, int32_t k2,
                            uint64_t seed, void* A_out, void* scratch, size_t scratch_bytes,
                            ts_stream stream);

/* ------------------------------------------------------------------------- */
/* Sketched rank-constrained least squares for one subproblem (Sec. 4, Alg. 5).
 *
 * Solves min ||Z B - Y||_F s.t. rank(B) <= R and returns B = CnT A^T with
 * CnT (r x R) and A (s x R, orthonormal columns).  Z is given COLUMN-major
 * (m x r, column c contiguous; the layout tensorsketch_apply writes), Y is
 * m x s row-major.  TS_SOLVE_RSVD runs Alg. 5 with the Gaussian test matrix of
 * (seed, TS_PURPOSE_RSVD_GAUSS, sweep, n) of k = max(R, min(R + oversample, r, s))
 * columns; TS_SOLVE_EXACT returns the best rank-R approximation of the
 * unconstrained solution.  Column signs: the largest-magnitude entry of each
 * column of A is positive (CnT flipped with it).
 * Errors: TS_ERR_SHAPE unless R <= min(r, s), r <= m, r <= 192 and k <= 64
 * (RSVD) or r <= 64 (EXACT); TS_ERR_NUMERIC is reported at the next
 * synchronising call if Z^T Z is not positive definite. */
size_t ts_lrls_scratch_bytes(int32_t m, int32_t r, int32_t s, int32_t R, int32_t solve,
                             int32_t oversample, int32_t dtype);
ts_status ts_lrls_solve(int32_t m, int32_t r, int32_t s, int32_t R, int32_t dtype,
                        const void* Z_colmajor, const void* Y, int32_t solve, uint64_t seed,
                        int32_t sweep, int32_t n, int32_t oversample, int32_t solve_fp64,
                        void* CnT_out, void* A_out, void* scratch, size_t scratch_bytes,
                        ts_stream stream);

/* ------------------------------------------------------------------------- */
/* Leverage-score sketch of subproblem `mode` of a dense or COO tensor (Sec. 3.2).
 *
 * For k != mode: l^(k)_i = sum_r A^(k)(i,r)^2 (ascending r, FP64), cdf by a
 * running FP64 sum in index order; sample j draws i_k = min{i : cdf_i > u cdf_last}
 * with u the uniform (seed, TS_PURPOSE_LEV_UNIFORM, sweep, mode, k; counter j).
 * Row j of Z (column-major m x prod R_k) is w_j (x)_k A^(k)(i_k, :) and row j of
 * Y (m x dims[mode]) is w_j T(i_{-mode}, :), w_j = 1/sqrt(m prod_k l_{i_k}/sum l).
 * factors: HOST array of X->order device pointers (entry `mode` ignored), each
 * dims[k] x ranks[k] in X's dtype.  samples_out (nullable): m x (order-1) int32,
 * the drawn i_k in ascending k.  Sampling uses the running-sum order above, so
 * for identical factor bits the samples are bit-identical to the oracle's.
 * COO input (Sec. 6 counts O(m s) for gathering the sampled fibres): the call first
 * builds, in the scratch, a hash index of the mode-`mode` fibres (keyed by the C-order
 * linear index of (i_k)_{k != mode}; capacity the power of two >= 2 nnz, about
 * 16 bytes per slot plus 4 + sizeof(value) per nonzero), then row j of Y is w_j times
 * the sum of the nonzeros of the sampled fibre at their mode coordinate (zero for an
 * empty fibre; repeated coordinates add, in an unspecified order).  Coordinates must
 * lie in [0, dims[k]); an out-of-range mode coordinate is dropped.
 * The int32 at offset 0 of the scratch is zeroed by the call and set non-zero if the
 * index could not place a nonzero (excluded by its capacity); read it after
 * synchronising.
 * Errors: TS_ERR_SHAPE for order > TS_MAX_ORDER or m < 1; TS_ERR_UNSUPPORTED for COO
 * input with >= 2^30 nonzeros or prod_{k != mode} dims[k] >= 9e18;
 * TS_ERR_WORKSPACE if scratch_bytes < ts_leverage_sketch_scratch_bytes(). */
size_t ts_leverage_sketch_scratch_bytes(const ts_tensor* X, int32_t mode, int32_t m);
ts_status ts_leverage_sketch(const ts_tensor* X, int32_t mode, const int32_t* ranks,
                             const void* const* factors, int32_t m, uint64_t seed, int32_t sweep,
                             void* Z_out, void* Y_out, int32_t* samples_out, void* scratch,
                             size_t scratch_bytes, ts_stream stream);

/* Deterministic leverage sketch ("Lev-fix", Sec. 3.2; kind TS_LEVERAGE_DET of
 * tucker_als_sketched): the min(m, C) multi-indices (i_k)_{k != mode} of largest score
 * prod_k l^(k)_{i_k} (C = prod_{k != mode} dims[k]; scores as above, products in FP64
 * rounded in ascending k), ties to the lower C-order linear index, in ascending linear
 * index; rows are not rescaled (weight 1), rows j >= C are zero.  Arguments, COO
 * handling and scratch as ts_leverage_sketch (no seed: nothing is drawn).
 * TS_ERR_UNSUPPORTED if C > 2^31 (every candidate is scored). */
ts_status ts_leverage_sketch_det(const ts_tensor* X, int32_t mode, const int32_t* ranks,
                                 const void* const* factors, int32_t m, void* Z_out, void* Y_out,
                                 int32_t* samples_out, void* scratch, size_t scratch_bytes,
                                 ts_stream stream);

/* ------------------------------------------------------------------------- */
/* Relative residual ||T - C x_1 A^(1) ... x_N A^(N)||_F / ||T||_F (Sec. 7 fitness
 * is 1 minus this).  Dense: direct reconstruction streamed against T with FP64
 * accumulation.  COO: ||T||^2 - 2<T, T~> + ||T~||^2 (clamped at 0) without forming
 * T~: ||T||^2 over distinct coordinates (repeated coordinates added first, through a
 * fibre index of the largest mode and a hash table of (fibre, coordinate) keys, both
 * in the scratch, about 56 bytes per nonzero), <T, T~> summed over the stored entries
 * with T~(i) formed in the data type, ||T~||^2 = <C, C x_1 G_1 ... x_N G_N> with
 * G_n = A^(n)T A^(n) (no orthonormality assumed); FP64 across entries.  The int32 at
 * offset 0 of the scratch is set non-zero if a hash table could not place an entry
 * (excluded by its capacity).
 * factors: HOST array of order device pointers (dims[k] x ranks[k]).
 * residual_out: DEVICE pointer to one double (0 when ||T|| = 0).
 * Errors: TS_ERR_UNSUPPORTED for COO input with order < 2, >= 2^30 nonzeros, the
 * product of the other dims of the largest mode >= 9e18, a core larger than 200 KB or
 * ranks[order-1] > 64. */
size_t ts_fitness_scratch_bytes(const ts_tensor* X, const int32_t* ranks);
ts_status ts_fitness(const ts_tensor* X, const int32_t* ranks, const void* core,
                     const void* const* factors, double* residual_out, void* scratch,
                     size_t scratch_bytes, ts_stream stream);

/* ------------------------------------------------------------------------- */
/* Sketch-Tucker-ALS (Alg. 4).
 *
 * Inputs: X, ranks (HOST, order entries), kind, sketch size m, sweeps >= 1.
 * Initialisation: Init-RRF for modes 1..N-1 (0-based) unless opt->init_given.
 * Each sweep updates modes 0..N-1 in order; subproblem n forms Z = S P^(n) and
 * Y = S T_(n)^T with TensorSketch (Y formed once and reused, or redrawn every
 * sweep with resketch_each_sweep), leverage-score sampling (redrawn every
 * subproblem) or deterministic leverage selection (TS_LEVERAGE_DET: the m rows of
 * largest score, reselected every subproblem), then solves it (opt->solve) and
 * writes A^(n) and the core.  Leverage sampling of a COO tensor builds the N fibre
 * indices of ts_leverage_sketch once, in the workspace, and gathers the sampled
 * fibres from them (< 2^30 nonzeros).
 * Outputs: core_out (prod ranks, C order), factors_inout (HOST array of order
 * device pointers, dims[k] x ranks[k]), residual_out (DEVICE, nullable):
 * `sweeps` doubles if opt->track_fit else one double, the final relative residual.
 * All outputs in X's dtype except residuals.
 * Numerical breakdown (a non-positive pivot of Z^T Z, a non-finite eigenvalue)
 * does not stop the enqueued work; it sets the int32 at offset 0 of the
 * workspace to a non-zero value (2: a COO fibre index could not place a nonzero,
 * excluded by its capacity), which the caller reads after synchronising.
 * Residuals of COO tensors follow ts_fitness (||T||^2 formed once per call, with its
 * fibre index and hash table in the workspace; TS_ERR_UNSUPPORTED under its limits).
 * tucker_als_workspace_bytes counts the residual's scratch whenever a residual can be
 * formed (for COO input about 56 bytes per nonzero), so one size serves calls with and
 * without residual_out.
 * Errors: TS_ERR_SHAPE if order < 2, any ranks[k] < 1 or ranks[k] >= dims[k]
 * (the theory assumes s > R), m < prod_{k != n} ranks[k] for some n (the sketched
 * system must be able to have full column rank), or a per-call limit above is
 * exceeded; TS_ERR_WORKSPACE if workspace_bytes < tucker_als_workspace_bytes(). */
ts_status tucker_als_workspace_bytes(const ts_tensor* X, const int32_t* ranks, int32_t kind,
                                     int32_t m, int32_t sweeps, const ts_options* opt,
                                     size_t* bytes_out);
ts_status tucker_als_sketched(const ts_tensor* X, const int32_t* ranks, int32_t kind, int32_t m,
                              int32_t sweeps, const ts_options* opt, void* workspace,
                              size_t workspace_bytes, void* core_out, void* const* factors_inout,
                              double* residual_out, ts_stream stream);

/* ------------------------------------------------------------------------- */
/* CP-Sketch-Tucker (Alg. 6): sketched Tucker-ALS to tucker_ranks, CP-ALS of rank
 * R_cp on the core (initialised by the HOSVD of the core, Sec. 7.2), CP factors
 * B^(n) A^(n) written to cp_factors_out (HOST array of order device pointers,
 * dims[k] x R_cp).  residual_out (DEVICE, nullable): one double, the relative
 * residual of the CP model against X.
 * Errors: as tucker_als_sketched, plus TS_ERR_SHAPE unless
 * R_cp <= min(tucker_ranks) and prod(tucker_ranks) <= 65536. */
ts_status cp_via_tucker_workspace_bytes(const ts_tensor* X, int32_t R_cp,
                                        const int32_t* tucker_ranks, int32_t m,
                                        int32_t tucker_sweeps, const ts_options* opt,
                                        size_t* bytes_out);
ts_status cp_via_tucker(const ts_tensor* X, int32_t R_cp, const int32_t* tucker_ranks, int32_t m,
                        int32_t tucker_sweeps, int32_t cp_sweeps, const ts_options* opt,
                        void* workspace, size_t workspace_bytes, void* const* cp_factors_out,
                        double* residual_out, ts_stream stream);

/* ------------------------------------------------------------------------- */
/* CP-ALS on a dense Tucker core: the inner step of Alg. 6 (CP decomposition of the
 * core produced by the sketched Tucker-ALS), exposed on its own so that it can be run
 * on any core.  The factors start from the HOSVD of the core (Sec. 7.2: the leading
 * R_cp left singular vectors of each unfolding, each column signed so that its
 * largest-magnitude entry is positive), then `sweeps` sweeps of Alg. 2 update every
 * factor by the normal equations: A^(n) = C_(n) KR_n (*_{k != n} A^(k)T A^(k))^{-1},
 * KR_n the Khatri-Rao product of the other factors (first factor slowest), the R_cp x
 * R_cp system solved in FP64 by Cholesky.  core: prod(ranks) values in C order (dtype
 * TS_F32 or TS_F64, DEVICE); factors_out: HOST array of `order` DEVICE pointers,
 * ranks[k] x R_cp row-major, overwritten.  R_cp <= min(ranks) (the HOSVD start).
 * Scratch: ts_cp_als_scratch_bytes (256-byte aligned); its first int32 is a device flag
 * set to non-zero when a Gram system is not positive definite (read it after the call).
 * Errors: TS_ERR_SHAPE for an order outside [2, TS_MAX_ORDER], non-positive ranks,
 * R_cp < 1 or R_cp > min(ranks), sweeps < 0; TS_ERR_WORKSPACE for short or misaligned
 * scratch. */
size_t ts_cp_als_scratch_bytes(int32_t order, const int32_t* ranks, int32_t R_cp, int32_t dtype);
ts_status ts_cp_als(int32_t order, const int32_t* ranks, int32_t R_cp, int32_t sweeps,
                    int32_t dtype, const void* core, void* const* factors_out, void* scratch,
                    size_t scratch_bytes, ts_stream stream);

/* ------------------------------------------------------------------------- */
/* Gradient of the sketched fit of subproblem `mode` (the objective that each step of
 * Alg. 4 minimises: eq. (tucker_ls) with the TensorSketch of Sec. 3.1 applied):
 *   L = 1/2 || Z C_(mode)^T A^(mode)T - Y ||_F^2,
 * Z = TensorSketch of the factors k != mode (tables[k], m buckets; columns in C order
 * of the remaining modes), C_(mode) the mode-`mode` unfolding of the core (C order),
 * Y (m x dims[mode], row-major) the sketched right-hand side, e.g. tensorsketch_input
 * with the same tables.  The factors k != mode enter through Z: their gradient is the
 * adjoint of the FFT chain (a circular cross-correlation per factor column) followed
 * by the transpose of each CountSketch (a hash/sign gather).
 * Inputs (all in `dtype`): core (prod ranks, C order), factors (HOST array of `order`
 * device pointers, dims[k] x ranks[k] row-major), tables (HOST array of `order` device
 * pointers, tables[mode] ignored), Y.  Outputs: loss (DEVICE, one double), grad_core
 * (prod ranks), grad_factors (HOST array of `order` device pointers, dims[k] x ranks[k]).
 * grad_core and grad_factors may both be NULL: then only the loss is computed (the
 * backward products and the adjoint of the FFT chain are skipped).
 * Errors: TS_ERR_SHAPE for an order outside [2, TS_MAX_ORDER], a mode out of range,
 * m outside [2, FFT limit] or non-positive sizes; TS_ERR_WORKSPACE for short or
 * misaligned scratch (ts_fit_grad_scratch_bytes; 0 for invalid shapes). */
size_t ts_fit_grad_scratch_bytes(int32_t order, const int64_t* dims, const int32_t* ranks,
                                 int32_t mode, int32_t m, int32_t dtype);
ts_status ts_fit_grad(int32_t order, const int64_t* dims, const int32_t* ranks, int32_t mode,
                      int32_t m, int32_t dtype, const void* core, const void* const* factors,
                      const int32_t* const* tables, const void* Y, double* loss,
                      void* grad_core, void* const* grad_factors, void* scratch,
                      size_t scratch_bytes, ts_stream stream);

/* ------------------------------------------------------------------------- */
/* Batched Sketch-Tucker-ALS: Alg. 4 on many independent dense tensors at once.
 *
 * Tensor i of `count` (X[i], HOST array of descriptors; one order N and dtype for the
 * batch) has ranks ranks[i*N .. i*N+N) (HOST), sketch size m[i] (HOST), and is
 * decomposed exactly as tucker_als_sketched decomposes it with the same options and
 * seed opt->seed + i (TensorSketch, Init-RRF unless opt->init_given, opt->solve); the
 * results equal that call's up to the summation order of the sketched products.
 * Every subproblem must fit the single-block solve (TS_ERR_UNSUPPORTED otherwise);
 * resketch_each_sweep, gram_bf16 and use_graph are not offered (TS_ERR_UNSUPPORTED).
 *
 * ts_batch_prepare: cores (HOST array of count device pointers, prod ranks, C order) and
 * factors (HOST array of count*N device pointers, tensor i's factor k at i*N + k,
 * dims[k] x ranks[k] row-major, holding the initial factors when opt->init_given) are
 * kept by the batch and updated in place by the sweeps.  Runs the setup of every
 * tensor (tables, the one-pass sketches, Init-RRF, the Gaussians of every sweep and
 * their products with the sketches), writes the per-subproblem launch descriptors into
 * the workspace, and times the product kernel with its two tile shapes on this batch
 * to keep the faster one per mode (the autotuner); synchronises `stream`.  *batch_out:
 * an opaque HOST handle, released with ts_batch_destroy (not before the work it
 * enqueued has finished).
 * ts_batch_sweeps: enqueues sweeps [first, first + nsweeps) of every tensor (in order;
 * sweep t uses the Gaussians of sweep t): per mode, four kernel launches over the whole
 * batch (factor CountSketch + FFT, Hadamard product + inverse FFT, the products
 * [Z^T Z | Z^T Y Omega | Z^T Y], the single-block solves); nothing else, so the call can
 * be captured in a CUDA graph.
 * ts_batch_residuals: residuals (DEVICE, count doubles) = the relative residual of each
 * tensor's current decomposition.
 * ts_batch_flags: flags_out (HOST, count int32) = each tensor's numerical-breakdown flag
 * (0: none); synchronous.
 * ts_batch_tiles: tiles_out (HOST, N int32) = the product tile kept per mode; ms_out
 * (HOST, 2N floats, nullable) = the measured times of tiles 32 and 64 per mode. */
typedef void* ts_batch;
ts_status ts_batch_workspace_bytes(int32_t count, const ts_tensor* X, const int32_t* ranks,
                                   const int32_t* m, int32_t sweeps, const ts_options* opt,
                                   size_t* bytes_out);
ts_status ts_batch_prepare(int32_t count, const ts_tensor* X, const int32_t* ranks,
                           const int32_t* m, int32_t sweeps, const ts_options* opt,
                           void* workspace, size_t workspace_bytes, void* const* cores,
                           void* const* factors, ts_batch* batch_out, ts_stream stream);
ts_status ts_batch_sweeps(ts_batch batch, int32_t first, int32_t nsweeps, ts_stream stream);
ts_status ts_batch_residuals(ts_batch batch, double* residuals, ts_stream stream);
ts_status ts_batch_flags(ts_batch batch, int32_t* flags_out);
ts_status ts_batch_tiles(ts_batch batch, int32_t* tiles_out, float* ms_out);
void ts_batch_destroy(ts_batch batch);

#ifdef __cplusplus
}
#endif

#endif /* TSKETCH_H */
