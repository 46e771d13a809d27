// Small dense linear algebra of the sketched rank-constrained solve (Sec. 4,
// Alg. 5).  Each kernel runs in ONE thread block with its operands in shared
// memory: the matrices are r x r (r = product of the other ranks) or k x k
// (k = R + oversampling), so the work is latency-bound and one SM keeps every
// intermediate on chip.  The design goal is few block-wide barriers: blocked
// Cholesky (16-wide panels factored by one warp with shuffles), blocked triangular
// solves, and a Jacobi eigensolver whose rotations of one round are applied by all
// threads at once (pair x column mapping, power-of-two strides).
//
// Precision.  The data type T is used throughout by default.  With `polish64`
// (FP32 data only) the QR of Alg. 5 runs in FP64 and the eigensolver ends with
// FP64 Jacobi sweeps on V^T K V: GB300's FP64 rate is ~1/64 of FP32, so this is an
// option, not the default.  FP64 data runs FP64 everywhere.
#include "dense_la.cuh"

namespace ts {

namespace {
constexpr int NT = 512;
constexpr int NWARP = NT / 32;
constexpr int NB = 16;  // Cholesky / triangular-solve panel width
}  // namespace


// ---------------------------------------------------------------- Cholesky

// In-place lower Cholesky of the r x r matrix at L (row stride ld, shared memory).
// A non-positive or non-finite pivot sets *flag and is replaced by 1.
template <typename T>
__device__ void chol_blocked(T* L, int r, int ld, int* flag) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarp = blockDim.x >> 5;
  for (int j0 = 0; j0 < r; j0 += NB) {
    const int nb = min(NB, r - j0);
    if (warp == 0) {  // diagonal block: lane i owns row j0 + i
      T row[NB];
      const bool mine = lane < nb;
#pragma unroll
      for (int c = 0; c < NB; ++c) row[c] = (mine && c < nb) ? L[(j0 + lane) * ld + j0 + c] : (T)0;
#pragma unroll
      for (int jj = 0; jj < NB; ++jj) {
        if (jj < nb) {
          T d = __shfl_sync(0xffffffffu, row[jj], jj);
          if (!(d > (T)0) || !isfinite((double)d)) {
            if (lane == 0 && flag) atomicExch(flag, 1);
            d = (T)1;
          }
          const T piv = sqrt(d);
          if (lane == jj) row[jj] = piv;
          if (lane > jj) row[jj] /= piv;
          const T lij = row[jj];
#pragma unroll
          for (int l = jj + 1; l < NB; ++l) {
            const T llj = __shfl_sync(0xffffffffu, row[jj], l);
            if (l < nb && lane >= l) row[l] -= lij * llj;
          }
        }
      }
      if (mine) {
#pragma unroll
        for (int c = 0; c < NB; ++c)
          if (c <= lane) L[(j0 + lane) * ld + j0 + c] = row[c];
      }
    }
    __syncthreads();
    // panel below the diagonal block: row i solves x L_dd^T = a
    for (int i = j0 + nb + threadIdx.x; i < r; i += blockDim.x) {
      T x[NB];
#pragma unroll
      for (int c = 0; c < NB; ++c) {
        if (c < nb) {
          T v = L[i * ld + j0 + c];
#pragma unroll
          for (int p = 0; p < c; ++p) v -= x[p] * L[(j0 + c) * ld + j0 + p];
          x[c] = v / L[(j0 + c) * ld + j0 + c];
        }
      }
#pragma unroll
      for (int c = 0; c < NB; ++c)
        if (c < nb) L[i * ld + j0 + c] = x[c];
    }
    __syncthreads();
    // trailing lower triangle: A(i, l) -= L(i, panel) L(l, panel)^T, l <= i
    const int t0 = j0 + nb;
    for (int ii = t0 + warp; ii < r; ii += nwarp) {
      for (int ll = t0 + lane; ll <= ii; ll += 32) {
        T acc = 0;
#pragma unroll
        for (int p = 0; p < NB; ++p)
          if (p < nb) acc += L[ii * ld + j0 + p] * L[ll * ld + j0 + p];
        L[ii * ld + ll] -= acc;
      }
    }
    __syncthreads();
  }
}

// B (r x k, row stride ldb) <- (L L^T)^{-1} B, blocked forward then backward substitution.
template <typename T>
__device__ void chol_solve_multi(const T* L, int r, int ld, T* B, int k, int ldb) {
  const int nblk = (r + NB - 1) / NB;
  for (int b = 0; b < nblk; ++b) {  // forward: L y = b
    const int j0 = b * NB, nb = min(NB, r - j0);
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
      for (int jj = 0; jj < nb; ++jj) {
        T v = B[(j0 + jj) * ldb + c];
        for (int p = 0; p < jj; ++p) v -= L[(j0 + jj) * ld + j0 + p] * B[(j0 + p) * ldb + c];
        B[(j0 + jj) * ldb + c] = v / L[(j0 + jj) * ld + j0 + jj];
      }
    }
    __syncthreads();
    const int rows = r - j0 - nb;
    for (int e = threadIdx.x; e < rows * k; e += blockDim.x) {
      const int i = j0 + nb + e / k, c = e % k;
      T acc = 0;
      for (int p = 0; p < nb; ++p) acc += L[i * ld + j0 + p] * B[(j0 + p) * ldb + c];
      B[i * ldb + c] -= acc;
    }
    __syncthreads();
  }
  for (int b = nblk - 1; b >= 0; --b) {  // backward: L^T x = y
    const int j0 = b * NB, nb = min(NB, r - j0);
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
      for (int jj = nb - 1; jj >= 0; --jj) {
        T v = B[(j0 + jj) * ldb + c];
        for (int p = jj + 1; p < nb; ++p) v -= L[(j0 + p) * ld + j0 + jj] * B[(j0 + p) * ldb + c];
        B[(j0 + jj) * ldb + c] = v / L[(j0 + jj) * ld + j0 + jj];
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < j0 * k; e += blockDim.x) {
      const int i = e / k, c = e % k;
      T acc = 0;
      for (int p = 0; p < nb; ++p) acc += L[(j0 + p) * ld + i] * B[(j0 + p) * ldb + c];
      B[i * ldb + c] -= acc;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- Householder QR

// Thin Householder QR of A (r x k, row stride k, r >= k) in compute type U: on exit
// Qo (r x k) holds orthonormal columns spanning range(A).  A zero column gives
// tau = 0 (identity reflector), so rank-deficient inputs are handled.
template <typename U>
__device__ void householder_q(U* A, int r, int k, U* Vh, U* tau, U* Qo, U* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarp = blockDim.x >> 5;
  for (int j = 0; j < k; ++j) {
    if (warp == 0) {
      U s = 0;
      for (int i = j + lane; i < r; i += 32) s += A[i * k + j] * A[i * k + j];
      s = warp_sum(s);
      if (lane == 0) {
        const U ajj = A[j * k + j];
        U tj = 0;
        red[0] = 0;
        if (s > (U)0) {
          const U alpha = ajj >= (U)0 ? -sqrt(s) : sqrt(s);
          const U v0 = ajj - alpha;
          const U vn2 = s - ajj * ajj + v0 * v0;
          tj = vn2 > (U)0 ? (U)2 / vn2 : (U)0;
          red[0] = v0;
        }
        tau[j] = tj;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < r; i += blockDim.x)
      Vh[i * k + j] = i < j ? (U)0 : (i == j ? red[0] : A[i * k + j]);
    __syncthreads();
    const U tj = tau[j];
    for (int c = j + 1 + warp; c < k; c += nwarp) {
      U w = 0;
      for (int i = j + lane; i < r; i += 32) w += Vh[i * k + j] * A[i * k + c];
      w = warp_sum(w) * tj;
      for (int i = j + lane; i < r; i += 32) A[i * k + c] -= w * Vh[i * k + j];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < r * k; t += blockDim.x) Qo[t] = (t / k == t % k) ? (U)1 : (U)0;
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    const U tj = tau[j];
    for (int c = warp; c < k; c += nwarp) {
      U w = 0;
      for (int i = j + lane; i < r; i += 32) w += Vh[i * k + j] * Qo[i * k + c];
      w = warp_sum(w) * tj;
      for (int i = j + lane; i < r; i += 32) Qo[i * k + c] -= w * Vh[i * k + j];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- RSVD-LRLS stage 1

size_t rsvd_stage1_smem_bytes(int r, int k, size_t tsize, bool qr64) {
  const size_t usize = qr64 ? 8 : tsize;
  return usize * (3 * (size_t)r * k + k + 2) + tsize * ((size_t)r * (r + 1) + (size_t)r * k) + 16;
}

// Alg. 5 up to the SVD: C = G^{-1} W, Q = qr(C), E = G^{-1} Q.  G and W are read
// with row strides ldg / ldw (they may be two column blocks of one product).
template <typename T, typename U>
__global__ void __launch_bounds__(NT) k_rsvd_stage1(int r, int k, const T* __restrict__ G,
                                                    int ldg, const T* __restrict__ W, int ldw,
                                                    T* __restrict__ Qout, T* __restrict__ Eout,
                                                    int* flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  U* A = reinterpret_cast<U*>(smem_raw);  // r x k
  U* Vh = A + r * k;                      // r x k
  U* Qd = Vh + r * k;                     // r x k
  U* tau = Qd + r * k;                    // k
  U* red = tau + k;                       // 2
  T* L = reinterpret_cast<T*>(red + 2);   // r x (r + 1)
  T* B = L + r * (r + 1);                 // r x k
  const int ld = r + 1;
  for (int i = threadIdx.x >> 5; i < r; i += NWARP)
    for (int j = threadIdx.x & 31; j <= i; j += 32) L[i * ld + j] = G[(long)i * ldg + j];
  for (int t = threadIdx.x; t < r * k; t += blockDim.x) B[t] = W[(long)(t / k) * ldw + t % k];
  __syncthreads();
  chol_blocked<T>(L, r, ld, flag);
  chol_solve_multi<T>(L, r, ld, B, k, k);
  for (int t = threadIdx.x; t < r * k; t += blockDim.x) A[t] = (U)B[t];
  __syncthreads();
  householder_q<U>(A, r, k, Vh, tau, Qd, red);
  for (int t = threadIdx.x; t < r * k; t += blockDim.x) {
    const T q = (T)Qd[t];
    Qout[t] = q;
    B[t] = q;
  }
  __syncthreads();
  chol_solve_multi<T>(L, r, ld, B, k, k);
  for (int t = threadIdx.x; t < r * k; t += blockDim.x) Eout[t] = B[t];
}

// Q = orth(C) for C (r x k) in one block (Householder in compute type U); used when r
// is too large for the on-chip Cholesky of stage 1.
template <typename T, typename U>
__global__ void __launch_bounds__(NT) k_qr_only(int r, int k, const T* __restrict__ C,
                                                T* __restrict__ Qout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  U* A = reinterpret_cast<U*>(smem_raw);  // r x k
  U* Vh = A + r * k;
  U* Qd = Vh + r * k;
  U* tau = Qd + r * k;
  U* red = tau + k;
  for (int t = threadIdx.x; t < r * k; t += blockDim.x) A[t] = (U)C[t];
  __syncthreads();
  householder_q<U>(A, r, k, Vh, tau, Qd, red);
  for (int t = threadIdx.x; t < r * k; t += blockDim.x) Qout[t] = (T)Qd[t];
}

// Newton-Schulz for G^{-1}: X0 = I / beta with beta the Gershgorin bound of lambda_max
// (max absolute row sum), so that ||I - G X0|| < 1 for SPD G.  First kernel: a warp per
// row, the row sums' maximum into *beta_bits (FP64 bits of a non-negative value: integer
// order is value order); second: X0 into X and 2I into twoI (the additive term of each
// iteration X <- X (2I - G X)).
template <typename T>
__global__ void k_ns_rowmax(int r, const T* __restrict__ G, long ldg,
                            unsigned long long* beta_bits) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= r) return;
  double srow = 0;
  for (int j = lane; j < r; j += 32) srow += fabs((double)G[(long)i * ldg + j]);
  for (int o = 16; o > 0; o >>= 1) srow += __shfl_xor_sync(0xffffffffu, srow, o);
  if (lane == 0) atomicMax(beta_bits, (unsigned long long)__double_as_longlong(srow));
}

template <typename T>
__global__ void k_ns_init(int r, const unsigned long long* __restrict__ beta_bits,
                          T* __restrict__ X, T* __restrict__ twoI) {
  const double beta = __longlong_as_double((long long)*beta_bits);
  const T inv = (T)(1.0 / (beta > 0 ? beta : 1.0));
  const long rr = (long)r * r;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < rr;
       e += (long)gridDim.x * blockDim.x) {
    const bool diag = (e / r) == (e % r);
    X[e] = diag ? inv : (T)0;
    twoI[e] = diag ? (T)2 : (T)0;
  }
}

template <typename T>
__global__ void k_copy(long n, const T* __restrict__ src, T* __restrict__ dst,
                       const int* skip = nullptr) {
  if (skip && *skip) return;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

// First launch of a Newton-Schulz step: S1 <- 2I, unless the iteration has stopped.
// conv[3] = "the previous step's check passed": that step's own update X <- X S1 has run,
// so from here on every launch returns (conv[0] = 1, read by the products and copies).
// All blocks read the same conv[3] (written by an earlier launch), so they agree.
template <typename T>
__global__ void k_ns_start(long n, const T* __restrict__ twoI, T* __restrict__ S1, int* conv) {
  if (conv[0]) return;
  if (conv[3]) {
    if (blockIdx.x == 0 && threadIdx.x == 0) conv[0] = 1;
    return;
  }
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    S1[e] = twoI[e];
}

// Newton-Schulz convergence: conv[3] = 1 once max |S1 - I| <= tol, S1 = 2I - G X, i.e.
// the residual E = I - G X of the current X is below tol entrywise.  The step's own update
// X <- X S1 = X (I + E) still runs and leaves a residual E^2 (quadratic convergence: at
// the rounding floor); the next step's k_ns_start turns conv[3] into the stop flag
// conv[0].  Blocks count their failures into conv[1]; the last block to finish (ticket
// conv[2]) decides and resets both counters.
template <typename T>
__global__ void k_ns_check(int r, const T* __restrict__ S1, int* conv, T tol) {
  __shared__ int bad;
  __shared__ bool last;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  if (conv[0] || conv[3]) return;  // uniform: every thread reads the same flags
  const long rr = (long)r * r;
  int mine = 0;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < rr;
       e += (long)gridDim.x * blockDim.x) {
    const T d = S1[e] - ((e / r) == (e % r) ? (T)1 : (T)0);
    mine |= !(fabs(d) <= tol);  // NaN counts as not converged
  }
  if (mine) atomicOr(&bad, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (bad) atomicAdd(conv + 1, 1);
    __threadfence();
    last = atomicAdd(conv + 2, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(conv + 1, 0) == 0) conv[3] = 1;
    conv[1] = 0;
    conv[2] = 0;
  }
}

template <typename T>
ts_status launch_qr_only(int r, int k, const T* C, T* Q, bool qr64, cudaStream_t st) {
  if (qr64 && sizeof(T) == 4) {
    const size_t smem = 8 * (3 * (size_t)r * k + k + 2);
    TS_TRY(ensure_dynamic_smem((const void*)k_qr_only<T, double>, smem));
    k_qr_only<T, double><<<1, NT, smem, st>>>(r, k, C, Q);
  } else {
    const size_t smem = sizeof(T) * (3 * (size_t)r * k + k + 2);
    TS_TRY(ensure_dynamic_smem((const void*)k_qr_only<T, T>, smem));
    k_qr_only<T, T><<<1, NT, smem, st>>>(r, k, C, Q);
  }
  TS_LAUNCH_CHECK();
  return TS_OK;
}

size_t qr_only_smem_bytes(int r, int k, bool qr64, size_t tsize) {
  return (qr64 ? 8 : tsize) * (3 * (size_t)r * k + k + 2);
}

// G^{-1} (r x r, into X) by `iters` Newton-Schulz steps; S1 holds 2 r^2 and S2 r^2 values.
template <typename T>
ts_status newton_schulz_inverse(int r, const T* G, long ldg, T* X, T* S1, T* S2, int iters,
                                int* conv, const GemmSplit<T>* split, cudaStream_t st) {
  const long rr = (long)r * r;
  // beta's bits live in S1 until the first iteration overwrites it
  unsigned long long* beta_bits = reinterpret_cast<unsigned long long*>(S1);
  TS_CUDA(cudaMemsetAsync(beta_bits, 0, sizeof(unsigned long long), st));
  k_ns_rowmax<T><<<ceil_div(r, 8), 256, 0, st>>>(r, G, ldg, beta_bits);
  TS_LAUNCH_CHECK();
  k_ns_init<T><<<ceil_div(rr, 256) > 1024 ? 1024 : ceil_div(rr, 256), 256, 0, st>>>(r, beta_bits,
                                                                                     X, S2);
  TS_LAUNCH_CHECK();
  // once the iteration has converged (k_ns_check, then the update of that step) the
  // remaining launches of the fixed schedule return at once: the schedule stays
  // graph-capturable.  conv holds 4 ints (stop flag, two counters, check passed).
  GemmSplit<T> sp = split ? *split : GemmSplit<T>{};
  sp.skip = conv;
  if (conv) TS_CUDA(cudaMemsetAsync(conv, 0, 4 * sizeof(int), st));
  const T tol = sizeof(T) == 4 ? (T)2e-6 : (T)1e-13;
  const int cb = ceil_div(rr, 256) > 1024 ? 1024 : ceil_div(rr, 256);
  const int chk = ceil_div(rr, 2048) > 256 ? 256 : ceil_div(rr, 2048);
  constexpr int kFirstCheck = 6;  // from a Gershgorin start the error halves at best early on
  for (int it = 0; it < iters; ++it) {
    // S1 = 2I - G X
    if (conv)
      k_ns_start<T><<<cb, 256, 0, st>>>(rr, S2, S1, conv);
    else
      k_copy<T><<<cb, 256, 0, st>>>(rr, S2, S1, nullptr);
    TS_LAUNCH_CHECK();
    TS_TRY(gemm<T>(r, r, r, -1.0, MatView<T>{G, ldg, 1}, MatView<T>{X, r, 1}, 1.0,
                   OutView<T>{S1, r, 1}, &sp, st));
    if (conv && it >= kFirstCheck) {
      k_ns_check<T><<<chk, 256, 0, st>>>(r, S1, conv, tol);
      TS_LAUNCH_CHECK();
    }
    // X <- X S1 (written through the first r*r of the split buffer)
    TS_TRY(gemm<T>(r, r, r, 1.0, MatView<T>{X, r, 1}, MatView<T>{S1, r, 1}, 0.0,
                   OutView<T>{S1 + rr, r, 1}, &sp, st));
    k_copy<T><<<cb, 256, 0, st>>>(rr, S1 + rr, X, conv);
    TS_LAUNCH_CHECK();
  }
  return TS_OK;
}

// ---------------------------------------------------------------- exact solve

// X = G^{-1} H, H r x s (row-major): one block, columns in chunks of 64.
template <typename T>
__global__ void __launch_bounds__(NT) k_chol_solve(int r, int s, const T* __restrict__ G,
                                                   const T* __restrict__ H, T* __restrict__ X,
                                                   int* flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* L = reinterpret_cast<T*>(smem_raw);  // r x (r + 1)
  T* B = L + r * (r + 1);                 // r x 64
  const int ld = r + 1;
  for (int i = threadIdx.x >> 5; i < r; i += NWARP)
    for (int j = threadIdx.x & 31; j <= i; j += 32) L[i * ld + j] = G[(long)i * r + j];
  __syncthreads();
  chol_blocked<T>(L, r, ld, flag);
  for (int c0 = 0; c0 < s; c0 += 64) {
    const int kc = min(64, s - c0);
    for (int t = threadIdx.x; t < r * kc; t += blockDim.x)
      B[(t / kc) * 64 + t % kc] = H[(long)(t / kc) * s + c0 + t % kc];
    __syncthreads();
    chol_solve_multi<T>(L, r, ld, B, kc, 64);
    for (int t = threadIdx.x; t < r * kc; t += blockDim.x)
      X[(long)(t / kc) * s + c0 + t % kc] = B[(t / kc) * 64 + t % kc];
    __syncthreads();
  }
}

// ---------------------------------------------------------------- symmetric eigensolver


// K (n x n) = U Lambda U^T, eigenvalues descending, sigma = sqrt(lambda):
// CnT = Q U_R Sigma_R (Q null: identity, r = n), Fm = U_R Sigma_R^{-1}, Uout = U_R.
template <typename T, bool POLISH64>
__global__ void __launch_bounds__(NT) k_eig_small(int n, int R, JacobiShape js,
                                                  const T* __restrict__ K,
                                                  const T* __restrict__ Q, int r,
                                                  T* __restrict__ CnT, T* __restrict__ Fm,
                                                  T* __restrict__ Uout, int* flag) {
  pdl_trigger();
  pdl_wait();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int rp[kMaxEig / 2 + 1], rq[kMaxEig / 2 + 1];
  __shared__ T rcT[kMaxEig / 2 + 1], rsT[kMaxEig / 2 + 1];
  __shared__ double rc64[POLISH64 ? kMaxEig / 2 + 1 : 1], rs64[POLISH64 ? kMaxEig / 2 + 1 : 1];
  __shared__ T redT[2 * NWARP + 2];
  __shared__ double red64[POLISH64 ? 2 * NWARP + 2 : 1];
  __shared__ int order[kMaxEig];
  __shared__ T lamT[kMaxEig];
  const int nn = n * n;
  T* A = reinterpret_cast<T*>(smem_raw);  // n x n
  T* V = A + nn;                          // n x n
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    const int i = e / n, j = e % n;
    A[e] = (T)0.5 * (K[i * n + j] + K[j * n + i]);
    V[e] = (i == j) ? (T)1 : (T)0;
  }
  __syncthreads();
  // stop on squared norms: off/tot cannot fall much below its rounding floor n^2 eps^2
  // (~1e-12 in FP32 at n = 8, ~6e-11 at n = 64), so the tolerance follows it for large n
  const T eps = sizeof(T) == 4 ? (T)1.1920929e-7 : (T)2.220446049250313e-16;
  const T floor4 = (T)4 * (T)n * (T)n * eps * eps;
  const T tol = sizeof(T) == 4 ? max((T)1e-11, floor4) : max((T)1e-28, floor4);
  T off, tot, prev = (T)-1;
  for (int sweep = 0; sweep < 24; ++sweep) {
    jacobi_norms<T>(A, n, redT, off, tot);
    if (off <= tol * tot || tot == (T)0) break;
    // a sweep that no longer cuts a small off-norm by 4x has met the rounding floor
    // (converging sweeps cut it quadratically)
    if (prev >= (T)0 && off <= (T)1e-6 * tot && off > (T)0.25 * prev) break;
    prev = off;
    jacobi_sweep<T>(A, V, js, rp, rq, rcT, rsT);
  }
  if constexpr (POLISH64) {
    // FP64 sweeps on V^T K V, V accumulated in FP64.
    double* A64 = reinterpret_cast<double*>(smem_raw + 2 * nn * sizeof(T) + 8 - ((2 * nn * sizeof(T)) & 7));
    double* V64 = A64 + nn;
    double* KV = V64 + nn;
    for (int e = threadIdx.x; e < nn; e += blockDim.x) V64[e] = (double)V[e];
    __syncthreads();
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
      const int i = e / n, j = e % n;
      double acc = 0;
      for (int b = 0; b < n; ++b)
        acc += 0.5 * ((double)K[i * n + b] + (double)K[b * n + i]) * V64[b * n + j];
      KV[e] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
      const int i = e / n, j = e % n;
      double acc = 0;
      for (int a = 0; a < n; ++a) acc += V64[a * n + i] * KV[a * n + j];
      A64[e] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
      const int i = e / n, j = e % n;
      if (i < j) {
        const double s = 0.5 * (A64[i * n + j] + A64[j * n + i]);
        A64[i * n + j] = s;
        A64[j * n + i] = s;
      }
    }
    __syncthreads();
    double o64, t64;
    for (int sweep = 0; sweep < 10; ++sweep) {
      jacobi_norms<double>(A64, n, red64, o64, t64);
      if (o64 <= 1e-28 * t64 || t64 == 0) break;
      jacobi_sweep<double>(A64, V64, js, rp, rq, rc64, rs64);
    }
    for (int e = threadIdx.x; e < nn; e += blockDim.x) V[e] = (T)V64[e];
    if (threadIdx.x < n) A[threadIdx.x * n + threadIdx.x] = (T)A64[threadIdx.x * n + threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < n; ++i) {
      lamT[i] = A[i * n + i];
      order[i] = i;
    }
    for (int i = 0; i < n; ++i) {  // selection sort, descending, stable on ties
      int best = i;
      for (int j = i + 1; j < n; ++j)
        if (lamT[order[j]] > lamT[order[best]]) best = j;
      const int t = order[i];
      order[i] = order[best];
      order[best] = t;
    }
    for (int i = 0; i < n; ++i)
      if (!isfinite((double)lamT[i]) && flag) atomicExch(flag, 1);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * R; e += blockDim.x) {
    const int i = e / R, c = e % R;
    const T l = lamT[order[c]];
    const T sig = l > (T)0 ? sqrt(l) : (T)0;
    const T u = V[i * n + order[c]];
    if (Fm) Fm[e] = sig > (T)0 ? u / sig : (T)0;
    if (Uout) Uout[e] = u;
  }
  if (CnT) {
    for (int e = threadIdx.x; e < r * R; e += blockDim.x) {
      const int i = e / R, c = e % R;
      const T l = lamT[order[c]];
      const T sig = l > (T)0 ? sqrt(l) : (T)0;
      T acc;
      if (Q) {
        acc = 0;
        for (int a = 0; a < n; ++a) acc += Q[i * n + a] * V[a * n + order[c]];
      } else {
        acc = V[i * n + order[c]];
      }
      CnT[e] = acc * sig;
    }
  }
}

// ---------------------------------------------------------------- signs, factor, core

// Column c of V = M Fm (M element (i, a) at M[i*rs + a*cs], a < kdim) or, with Fm
// null, V(i, c) = M[i*rs + c*cs].
template <typename T>
__device__ __forceinline__ T vcol(const T* M, long rs, long cs, int kdim, const T* Fm, int R,
                                  int i, int c) {
  if (!Fm) return M[i * rs + c * cs];
  T v = 0;
  for (int a = 0; a < kdim; ++a) v += M[i * rs + a * cs] * Fm[a * R + c];
  return v;
}

// Column c of C_(n)^T flipped by sgn and, when core != null, scattered into the core.
template <typename T>
__device__ __forceinline__ void flip_core_column(int c, int R, T sgn, T* __restrict__ CnT, int r,
                                                 T* __restrict__ core, const CoreMap& map) {
  for (int rho = threadIdx.x; rho < r; rho += blockDim.x) {
    const T v = sgn * CnT[(long)rho * R + c];
    CnT[(long)rho * R + c] = v;
    if (core) {
      long idx = 0, stride = 1, x = rho;
      for (int k = map.order - 1; k >= 0; --k) {
        int digit;
        if (k == map.n) {
          digit = c;
        } else {
          digit = (int)(x % map.ranks[k]);
          x /= map.ranks[k];
        }
        idx += digit * stride;
        stride *= map.ranks[k];
      }
      core[idx] = v;
    }
  }
}

// (value, index) of the larger magnitude, the lower index on ties
template <typename T>
__device__ __forceinline__ void keep_larger(T& bv, int& bi, T v, int i) {
  if (v > bv || (v == bv && i < bi)) {
    bv = v;
    bi = i;
  }
}

template <typename T>
__device__ __forceinline__ void block_argmax(T& best, int& bidx, T* bv, int* bi) {
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = bidx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) keep_larger(bv[threadIdx.x], bi[threadIdx.x], bv[threadIdx.x + w],
                                     bi[threadIdx.x + w]);
    __syncthreads();
  }
  best = bv[0];
  bidx = bi[0];
}

// Block c: canonical sign of column c of V (entry of largest magnitude positive,
// lowest index on ties); A_out(:, c) = sign * V(:, c), CnT(:, c) *= sign and, when
// core != null, C_(n)^T is scattered into the core.
template <typename T>
__global__ void __launch_bounds__(256) k_finalize(int s, int R, const T* __restrict__ M, long rs,
                                                  long cs, int kdim, const T* __restrict__ Fm,
                                                  T* __restrict__ A_out, T* __restrict__ CnT,
                                                  int r, T* __restrict__ core, CoreMap map) {
  pdl_trigger();
  pdl_wait();
  __shared__ T bv[256];
  __shared__ int bi[256];
  const int c = blockIdx.x;
  T best = (T)-1;
  int bidx = 0x7fffffff;
  for (int i = threadIdx.x; i < s; i += blockDim.x)
    keep_larger(best, bidx, (T)fabs(vcol<T>(M, rs, cs, kdim, Fm, R, i, c)), i);
  block_argmax(best, bidx, bv, bi);
  const T sgn = vcol<T>(M, rs, cs, kdim, Fm, R, bidx, c) < (T)0 ? (T)-1 : (T)1;
  for (int i = threadIdx.x; i < s; i += blockDim.x)
    A_out[(long)i * R + c] = sgn * vcol<T>(M, rs, cs, kdim, Fm, R, i, c);
  if (CnT) flip_core_column(c, R, sgn, CnT, r, core, map);
}

// Tall columns, first pass: block (b, c) finds the largest |V(i, c)| over its chunk of rows.
template <typename T>
__global__ void __launch_bounds__(256) k_finalize_scan(int s, int R, const T* __restrict__ M,
                                                       long rs, long cs, int kdim,
                                                       const T* __restrict__ Fm, int chunk,
                                                       T* __restrict__ pv, int* __restrict__ pi) {
  pdl_trigger();
  pdl_wait();
  __shared__ T bv[256];
  __shared__ int bi[256];
  const int c = blockIdx.y, b = blockIdx.x;
  const int i1 = min(s, (b + 1) * chunk);
  T best = (T)-1;
  int bidx = 0x7fffffff;
  for (int i = b * chunk + threadIdx.x; i < i1; i += blockDim.x)
    keep_larger(best, bidx, (T)fabs(vcol<T>(M, rs, cs, kdim, Fm, R, i, c)), i);
  block_argmax(best, bidx, bv, bi);
  if (threadIdx.x == 0) {
    pv[(long)c * gridDim.x + b] = best;
    pi[(long)c * gridDim.x + b] = bidx;
  }
}

// Second pass: every block reduces the column's chunk maxima (the same winner as the
// one-block pass), writes its chunk of A_out; block (0, c) flips C_(n)^T.
template <typename T>
__global__ void __launch_bounds__(256) k_finalize_write(int s, int R, const T* __restrict__ M,
                                                        long rs, long cs, int kdim,
                                                        const T* __restrict__ Fm, int chunk,
                                                        const T* __restrict__ pv,
                                                        const int* __restrict__ pi,
                                                        T* __restrict__ A_out, T* __restrict__ CnT,
                                                        int r, T* __restrict__ core, CoreMap map) {
  pdl_trigger();
  pdl_wait();
  __shared__ T bv[256];
  __shared__ int bi[256];
  const int c = blockIdx.y, b = blockIdx.x, nb = gridDim.x;
  T best = (T)-1;
  int bidx = 0x7fffffff;
  for (int j = threadIdx.x; j < nb; j += blockDim.x)
    keep_larger(best, bidx, pv[(long)c * nb + j], pi[(long)c * nb + j]);
  block_argmax(best, bidx, bv, bi);
  const T sgn = vcol<T>(M, rs, cs, kdim, Fm, R, bidx, c) < (T)0 ? (T)-1 : (T)1;
  const int i1 = min(s, (b + 1) * chunk);
  for (int i = b * chunk + threadIdx.x; i < i1; i += blockDim.x)
    A_out[(long)i * R + c] = sgn * vcol<T>(M, rs, cs, kdim, Fm, R, i, c);
  if (CnT && b == 0) flip_core_column(c, R, sgn, CnT, r, core, map);
}

// ---------------------------------------------------------------- launchers

template <typename T>
ts_status launch_rsvd_stage1(int r, int k, const T* G, int ldg, const T* W, int ldw, T* Q, T* E,
                             bool qr64, int* flag, cudaStream_t st) {
  if (qr64 && sizeof(T) == 4) {
    const size_t smem = rsvd_stage1_smem_bytes(r, k, sizeof(T), true);
    TS_TRY(ensure_dynamic_smem((const void*)k_rsvd_stage1<T, double>, smem));
    k_rsvd_stage1<T, double><<<1, NT, smem, st>>>(r, k, G, ldg, W, ldw, Q, E, flag);
  } else {
    const size_t smem = rsvd_stage1_smem_bytes(r, k, sizeof(T), false);
    TS_TRY(ensure_dynamic_smem((const void*)k_rsvd_stage1<T, T>, smem));
    k_rsvd_stage1<T, T><<<1, NT, smem, st>>>(r, k, G, ldg, W, ldw, Q, E, flag);
  }
  TS_LAUNCH_CHECK();
  return TS_OK;
}

size_t chol_solve_smem_bytes(int r, size_t tsize) {
  return tsize * ((size_t)r * (r + 1) + (size_t)r * 64);
}

template <typename T>
ts_status launch_chol_solve(int r, int s, const T* G, const T* H, T* X, int* flag,
                            cudaStream_t st) {
  const size_t smem = chol_solve_smem_bytes(r, sizeof(T));
  TS_TRY(ensure_dynamic_smem((const void*)k_chol_solve<T>, smem));
  k_chol_solve<T><<<1, NT, smem, st>>>(r, s, G, H, X, flag);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

template <typename T>
ts_status launch_eig_small(int n, int R, const T* K, const T* Q, int r, T* CnT, T* Fm, T* Uout,
                           bool polish64, int* flag, cudaStream_t st) {
  if (n > kMaxEig || n < 1)
    return fail(TS_ERR_SHAPE, "eigensolver: n=%d outside [1,%d]", n, kMaxEig);
  if (n <= 16 && R <= n)  // four-warp Jacobi on an 8-CTA cluster (lrls_chol.cu)
    return launch_eig16<T>(n, R, K, Q, r, CnT, Fm, Uout, polish64, flag, st);
  JacobiShape js;
  js.n = n;
  js.np = (n + 1) & ~1;
  js.lg = 0;
  while ((1 << js.lg) < n) ++js.lg;
  const int work = (js.np / 2) << js.lg;
  int threads = work < NT ? ((work + 31) / 32) * 32 : NT;
  if (threads < 64) threads = 64;
  const size_t nn = (size_t)n * n;
  if (polish64 && sizeof(T) == 4) {
    const size_t smem = nn * 2 * sizeof(T) + 8 + nn * 3 * sizeof(double);
    TS_TRY(ensure_dynamic_smem((const void*)k_eig_small<T, true>, smem));
    TS_TRY(launch_pdl(k_eig_small<T, true>, dim3(1), dim3(threads), smem, st, n, R, js, K, Q, r,
                      CnT, Fm, Uout, flag));
  } else {
    const size_t smem = nn * 2 * sizeof(T);
    TS_TRY(ensure_dynamic_smem((const void*)k_eig_small<T, false>, smem));
    TS_TRY(launch_pdl(k_eig_small<T, false>, dim3(1), dim3(threads), smem, st, n, R, js, K, Q, r,
                      CnT, Fm, Uout, flag));
  }
  TS_LAUNCH_CHECK();
  return TS_OK;
}

template <typename T>
ts_status launch_finalize(int s, int R, const T* M, long rs, long cs, int kdim, const T* Fm,
                          T* A_out, T* CnT, int r, T* core, CoreMap map, cudaStream_t st,
                          void* scratch, size_t scratch_bytes) {
  // tall columns over many SMs when the caller lends scratch for the chunk maxima
  const int chunk = std::max(2048, ceil_div(s, 256));
  const int nb = ceil_div(s, chunk);
  if (nb >= 4 && scratch &&
      scratch_bytes >= (size_t)nb * R * (sizeof(T) + sizeof(int)) + 256) {
    T* pv = static_cast<T*>(scratch);
    int* pi = reinterpret_cast<int*>(static_cast<char*>(scratch) +
                                     align_up((size_t)nb * R * sizeof(T), 256));
    TS_TRY(launch_pdl(k_finalize_scan<T>, dim3(nb, R), dim3(256), 0, st, s, R, M, rs, cs, kdim,
                      Fm, chunk, pv, pi));
    return launch_pdl(k_finalize_write<T>, dim3(nb, R), dim3(256), 0, st, s, R, M, rs, cs, kdim,
                      Fm, chunk, (const T*)pv, (const int*)pi, A_out, CnT, r, core, map);
  }
  return launch_pdl(k_finalize<T>, dim3(R), dim3(256), 0, st, s, R, M, rs, cs, kdim, Fm, A_out,
                    CnT, r, core, map);
}

#define TS_INST(T)                                                                               \
  template ts_status launch_rsvd_stage1<T>(int, int, const T*, int, const T*, int, T*, T*, bool, \
                                           int*, cudaStream_t);                                  \
  template ts_status launch_chol_solve<T>(int, int, const T*, const T*, T*, int*, cudaStream_t); \
  template ts_status launch_eig_small<T>(int, int, const T*, const T*, int, T*, T*, T*, bool,   \
                                         int*, cudaStream_t);                                    \
  template ts_status launch_finalize<T>(int, int, const T*, long, long, int, const T*, T*, T*,  \
                                        int, T*, CoreMap, cudaStream_t, void*, size_t);          \
  template ts_status launch_qr_only<T>(int, int, const T*, T*, bool, cudaStream_t);             \
  template ts_status newton_schulz_inverse<T>(int, const T*, long, T*, T*, T*, int, int*,       \
                                              const GemmSplit<T>*, cudaStream_t);
TS_INST(float)
TS_INST(double)
#undef TS_INST

}  // namespace ts
