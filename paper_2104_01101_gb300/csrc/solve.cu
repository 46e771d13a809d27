// Small dense linear algebra of the sketched rank-constrained solve (Sec. 4,
// Alg. 5).  Every kernel here runs in ONE thread block with its operands in
// shared memory: the matrices are r x r (r = prod of the other ranks, <= 192)
// or k x k (k = R + oversampling, <= 64), so the work is latency-bound and a
// single SM keeps every intermediate on chip.
//
// Precision: Cholesky of Z^T Z and the triangular solves run in the data type T;
// the QR of Alg. 5 (Householder) runs in FP64; the symmetric eigensolver that
// yields the SVD runs Jacobi sweeps in T and finishes with FP64 sweeps.
#include "internal.cuh"

namespace ts {

namespace {
constexpr int NT = 512;
constexpr int NWARP = NT / 32;
}  // namespace

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// In-place lower Cholesky of the r x r matrix in shared memory (row stride r).
// Sets *flag = 1 (and substitutes 1 for the pivot) if a pivot is not positive.
template <typename T>
__device__ void chol_smem(T* L, int r, int* flag) {
  for (int j = 0; j < r; ++j) {
    if (threadIdx.x == 0) {
      T d = L[j * r + j];
      if (!(d > (T)0) || !isfinite((double)d)) {
        if (flag) atomicExch(flag, 1);
        d = (T)1;
      }
      L[j * r + j] = sqrt(d);
    }
    __syncthreads();
    const T piv = L[j * r + j];
    for (int i = j + 1 + threadIdx.x; i < r; i += blockDim.x) L[i * r + j] /= piv;
    __syncthreads();
    const int n = r - j - 1;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
      const int i = j + 1 + t / n, l = j + 1 + t % n;
      if (l <= i) L[i * r + l] -= L[i * r + j] * L[l * r + j];
    }
    __syncthreads();
  }
}

// Solve (L L^T) x = b in place for column `col` of B (r x ncols, row stride ld),
// one warp per column.
template <typename T>
__device__ void chol_solve_col_warp(const T* L, int r, T* B, int ld, int col) {
  const int lane = threadIdx.x & 31;
  for (int i = 0; i < r; ++i) {
    T part = 0;
    for (int l = lane; l < i; l += 32) part += L[i * r + l] * B[l * ld + col];
    part = warp_sum(part);
    if (lane == 0) B[i * ld + col] = (B[i * ld + col] - part) / L[i * r + i];
    __syncwarp();
  }
  for (int i = r - 1; i >= 0; --i) {
    T part = 0;
    for (int l = i + 1 + lane; l < r; l += 32) part += L[l * r + i] * B[l * ld + col];
    part = warp_sum(part);
    if (lane == 0) B[i * ld + col] = (B[i * ld + col] - part) / L[i * r + i];
    __syncwarp();
  }
}

// Thin Householder QR of A (r x k, FP64, row stride k, r >= k) in shared memory:
// on exit Qo (r x k) holds the orthonormal factor.  Vh (r x k) and tau (k) are
// work arrays.  Robust to rank deficiency (a zero column gives tau = 0).
__device__ void householder_q(double* A, int r, int k, double* Vh, double* tau, double* Qo,
                              double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = 0; j < k; ++j) {
    if (warp == 0) {
      double s = 0;
      for (int i = j + lane; i < r; i += 32) s += A[i * k + j] * A[i * k + j];
      s = warp_sum(s);
      if (lane == 0) {
        const double ajj = A[j * k + j];
        double tj = 0;
        if (s > 0) {
          const double alpha = ajj >= 0 ? -sqrt(s) : sqrt(s);
          const double v0 = ajj - alpha;
          const double vn2 = s - ajj * ajj + v0 * v0;
          tj = vn2 > 0 ? 2.0 / vn2 : 0.0;
          red[0] = v0;
          red[1] = alpha;
        } else {
          red[0] = 0;
          red[1] = ajj;
        }
        tau[j] = tj;
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < r; i += blockDim.x)
      Vh[i * k + j] = i < j ? 0.0 : (i == j ? red[0] : A[i * k + j]);
    __syncthreads();
    const double tj = tau[j];
    for (int c = j + 1 + warp; c < k; c += NWARP) {
      double w = 0;
      for (int i = j + lane; i < r; i += 32) w += Vh[i * k + j] * A[i * k + c];
      w = warp_sum(w) * tj;
      for (int i = j + lane; i < r; i += 32) A[i * k + c] -= w * Vh[i * k + j];
    }
    __syncthreads();
  }
  // Q = H_0 ... H_{k-1} [I; 0], applied from the last reflector.
  for (int t = threadIdx.x; t < r * k; t += blockDim.x) Qo[t] = (t / k == t % k) ? 1.0 : 0.0;
  __syncthreads();
  for (int j = k - 1; j >= 0; --j) {
    const double tj = tau[j];
    for (int c = warp; c < k; c += NWARP) {
      double w = 0;
      for (int i = j + lane; i < r; i += 32) w += Vh[i * k + j] * Qo[i * k + c];
      w = warp_sum(w) * tj;
      for (int i = j + lane; i < r; i += 32) Qo[i * k + c] -= w * Vh[i * k + j];
    }
    __syncthreads();
  }
}

// Alg. 5 up to the SVD: C = G^{-1} W, Q = qr(C), E = G^{-1} Q.
template <typename T>
__global__ void __launch_bounds__(NT) k_rsvd_stage1(int r, int k, const T* __restrict__ G,
                                                    const T* __restrict__ W, T* __restrict__ Qout,
                                                    T* __restrict__ Eout, int* flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* A = reinterpret_cast<double*>(smem_raw);  // r x k
  double* Vh = A + r * k;                           // r x k
  double* Qd = Vh + r * k;                          // r x k
  double* tau = Qd + r * k;                         // k
  double* red = tau + k;                            // 2
  T* L = reinterpret_cast<T*>(red + 2);             // r x r
  T* B = L + r * r;                                 // r x k
  for (int t = threadIdx.x; t < r * r; t += blockDim.x) L[t] = G[t];
  for (int t = threadIdx.x; t < r * k; t += blockDim.x) B[t] = W[t];
  __syncthreads();
  chol_smem<T>(L, r, flag);
  const int warp = threadIdx.x >> 5;
  for (int c = warp; c < k; c += NWARP) chol_solve_col_warp<T>(L, r, B, k, c);
  __syncthreads();
  for (int t = threadIdx.x; t < r * k; t += blockDim.x) A[t] = (double)B[t];
  __syncthreads();
  householder_q(A, r, k, Vh, tau, Qd, red);
  for (int t = threadIdx.x; t < r * k; t += blockDim.x) {
    const T q = (T)Qd[t];
    Qout[t] = q;
    B[t] = q;
  }
  __syncthreads();
  for (int c = warp; c < k; c += NWARP) chol_solve_col_warp<T>(L, r, B, k, c);
  __syncthreads();
  for (int t = threadIdx.x; t < r * k; t += blockDim.x) Eout[t] = B[t];
}

// X = G^{-1} H, H r x s (row-major), all columns in one block.
template <typename T>
__global__ void __launch_bounds__(NT) k_chol_solve(int r, int s, const T* __restrict__ G,
                                                   const T* __restrict__ H, T* __restrict__ X,
                                                   int* flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* L = reinterpret_cast<T*>(smem_raw);  // r x r
  T* Bw = L + r * r;                      // NWARP x r  (one column per warp)
  for (int t = threadIdx.x; t < r * r; t += blockDim.x) L[t] = G[t];
  __syncthreads();
  chol_smem<T>(L, r, flag);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* b = Bw + warp * r;
  for (int c = warp; c < s; c += NWARP) {
    for (int i = lane; i < r; i += 32) b[i] = H[(long)i * s + c];
    __syncwarp();
    chol_solve_col_warp<T>(L, r, b, 1, 0);
    for (int i = lane; i < r; i += 32) X[(long)i * s + c] = b[i];
    __syncwarp();
  }
}

// One cyclic Jacobi sweep (round-robin pairing, n padded to even) on the n x n
// symmetric matrix A with accumulated eigenvectors V; returns nothing, caller checks.
template <typename U>
__device__ void jacobi_sweep(U* A, U* V, int n, int* rp, int* rq, U* rc, U* rs) {
  const int np = (n + 1) & ~1;
  const int npairs = np / 2;
  for (int t = 0; t < np - 1; ++t) {
    if (threadIdx.x < npairs) {
      const int i = threadIdx.x;
      int a, b;
      if (i == 0) {
        a = t;
        b = np - 1;
      } else {
        a = (t + i) % (np - 1);
        b = (t - i + np - 1) % (np - 1);
      }
      int p = a < b ? a : b, q = a < b ? b : a;
      U c = 1, s = 0;
      if (q < n) {
        const U apq = A[p * n + q];
        if (apq != (U)0) {
          const U theta = (A[q * n + q] - A[p * n + p]) / (2 * apq);
          const U tt = (theta >= 0 ? (U)1 : (U)-1) / (fabs(theta) + sqrt(theta * theta + (U)1));
          c = (U)1 / sqrt(tt * tt + (U)1);
          s = tt * c;
        }
      } else {
        p = q = -1;
      }
      rp[i] = p;
      rq[i] = q;
      rc[i] = c;
      rs[i] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < npairs * n; e += blockDim.x) {
      const int i = e / n, l = e % n;
      const int p = rp[i], q = rq[i];
      if (p < 0) continue;
      const U c = rc[i], s = rs[i];
      const U ap = A[p * n + l], aq = A[q * n + l];
      A[p * n + l] = c * ap - s * aq;
      A[q * n + l] = s * ap + c * aq;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < npairs * n; e += blockDim.x) {
      const int i = e / n, l = e % n;
      const int p = rp[i], q = rq[i];
      if (p < 0) continue;
      const U c = rc[i], s = rs[i];
      const U ap = A[l * n + p], aq = A[l * n + q];
      A[l * n + p] = c * ap - s * aq;
      A[l * n + q] = s * ap + c * aq;
      const U vp = V[l * n + p], vq = V[l * n + q];
      V[l * n + p] = c * vp - s * vq;
      V[l * n + q] = s * vp + c * vq;
    }
    __syncthreads();
  }
}

// Returns off-diagonal^2 and total^2 of A (block-wide; result valid in all threads).
template <typename U>
__device__ void offdiag_norms(const U* A, int n, double* red, double& off, double& tot) {
  double o = 0, a = 0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const double v = (double)A[e];
    a += v * v;
    if (e / n != e % n) o += v * v;
  }
  o = warp_sum(o);
  a = warp_sum(a);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[2 * warp] = o;
    red[2 * warp + 1] = a;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double so = 0, sa = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      so += red[2 * w];
      sa += red[2 * w + 1];
    }
    red[2 * NWARP] = so;
    red[2 * NWARP + 1] = sa;
  }
  __syncthreads();
  off = red[2 * NWARP];
  tot = red[2 * NWARP + 1];
  __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(NT) k_eig_small(int n, int R, const T* __restrict__ K,
                                                  const T* __restrict__ Q, int r,
                                                  T* __restrict__ CnT, T* __restrict__ Fm,
                                                  T* __restrict__ Uout, int* flag) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int rp[kMaxEig / 2 + 1], rq[kMaxEig / 2 + 1];
  __shared__ double rc64[kMaxEig / 2 + 1], rs64[kMaxEig / 2 + 1];
  __shared__ T rc32[kMaxEig / 2 + 1], rs32[kMaxEig / 2 + 1];
  __shared__ double red[2 * NWARP + 2];
  __shared__ int order[kMaxEig];
  __shared__ double lam[kMaxEig];
  const int nn = n * n;
  double* A64 = reinterpret_cast<double*>(smem_raw);  // n x n
  double* V64 = A64 + nn;                             // n x n
  double* K64 = V64 + nn;                             // n x n
  T* A32 = reinterpret_cast<T*>(K64 + nn);            // n x n
  T* V32 = A32 + nn;                                  // n x n
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    const int i = e / n, j = e % n;
    const T sym = (T)0.5 * (K[i * n + j] + K[j * n + i]);
    A32[e] = sym;
    K64[e] = (double)sym;
    V32[e] = (i == j) ? (T)1 : (T)0;
  }
  __syncthreads();
  double off, tot;
  // Phase 1: Jacobi sweeps in the data type (skipped for FP64 data).
  if (sizeof(T) == 4) {
    for (int sweep = 0; sweep < 30; ++sweep) {
      offdiag_norms<T>(A32, n, red, off, tot);
      if (off <= 1e-12 * tot || tot == 0) break;
      jacobi_sweep<T>(A32, V32, n, rp, rq, rc32, rs32);
    }
  }
  // Phase 2: FP64 sweeps on V^T K V (K V into A64, then V^T (K V) into K64).
  for (int e = threadIdx.x; e < nn; e += blockDim.x) V64[e] = (double)V32[e];
  __syncthreads();
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    const int i = e / n, j = e % n;
    double acc = 0;
    for (int b = 0; b < n; ++b) acc += K64[i * n + b] * V64[b * n + j];
    A64[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    const int i = e / n, j = e % n;
    double acc = 0;
    for (int a = 0; a < n; ++a) acc += V64[a * n + i] * A64[a * n + j];
    K64[e] = acc;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    const int i = e / n, j = e % n;
    A64[e] = 0.5 * (K64[i * n + j] + K64[j * n + i]);
  }
  __syncthreads();
  for (int sweep = 0; sweep < 30; ++sweep) {
    offdiag_norms<double>(A64, n, red, off, tot);
    if (off <= 1e-28 * tot || tot == 0) break;
    jacobi_sweep<double>(A64, V64, n, rp, rq, rc64, rs64);
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < n; ++i) {
      lam[i] = A64[i * n + i];
      order[i] = i;
    }
    for (int i = 0; i < n; ++i) {  // selection sort, descending, stable on ties
      int best = i;
      for (int j = i + 1; j < n; ++j)
        if (lam[order[j]] > lam[order[best]]) best = j;
      const int t = order[i];
      order[i] = order[best];
      order[best] = t;
    }
    for (int i = 0; i < n; ++i)
      if (!isfinite(lam[i]) && flag) atomicExch(flag, 1);
  }
  __syncthreads();
  // Fm = U_R Sigma_R^{-1}, Uout = U_R
  for (int e = threadIdx.x; e < n * R; e += blockDim.x) {
    const int i = e / R, c = e % R;
    const double l = lam[order[c]];
    const double sig = l > 0 ? sqrt(l) : 0.0;
    if (Fm) Fm[e] = (T)(sig > 0 ? V64[i * n + order[c]] / sig : 0.0);
    if (Uout) Uout[e] = (T)V64[i * n + order[c]];
  }
  // CnT = Q U_R Sigma_R
  if (CnT) for (int e = threadIdx.x; e < r * R; e += blockDim.x) {
    const int i = e / R, c = e % R;
    const double l = lam[order[c]];
    const double sig = l > 0 ? sqrt(l) : 0.0;
    double acc;
    if (Q) {
      acc = 0;
      for (int a = 0; a < n; ++a) acc += (double)Q[i * n + a] * V64[a * n + order[c]];
    } else {
      acc = V64[i * n + order[c]];
    }
    CnT[e] = (T)(acc * sig);
  }
}

// Block c: canonical sign of column c of V (largest |.|, lowest index on ties).
template <typename T>
__global__ void __launch_bounds__(256) k_finalize(int s, int R, const T* V, T* A_out, T* CnT,
                                                  int r, T* core, CoreMap map) {
  __shared__ double bv[256];
  __shared__ int bi[256];
  const int c = blockIdx.x;
  double best = -1.0;
  int bidx = 0x7fffffff;
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    const double a = fabs((double)V[(long)i * R + c]);
    if (a > best || (a == best && i < bidx)) {
      best = a;
      bidx = i;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = bidx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      const double ob = bv[threadIdx.x + w];
      const int oi = bi[threadIdx.x + w];
      if (ob > bv[threadIdx.x] || (ob == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
        bv[threadIdx.x] = ob;
        bi[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const T sgn = V[(long)bi[0] * R + c] < (T)0 ? (T)-1 : (T)1;
  __syncthreads();
  for (int i = threadIdx.x; i < s; i += blockDim.x) A_out[(long)i * R + c] = sgn * V[(long)i * R + c];
  if (CnT) {
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
}

static ts_status smem_attr(const void* fn, size_t bytes) {
  if (bytes > kMaxSmem) return fail(TS_ERR_SHAPE, "shared-memory footprint %zu too large", bytes);
  if (bytes > 48 * 1024)
    TS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return TS_OK;
}

template <typename T>
ts_status launch_rsvd_stage1(int r, int k, const T* G, const T* W, T* Q, T* E, int* flag,
                             cudaStream_t st) {
  const size_t smem = rsvd_stage1_smem_bytes(r, k, sizeof(T));
  TS_TRY(smem_attr((const void*)k_rsvd_stage1<T>, smem));
  k_rsvd_stage1<T><<<1, NT, smem, st>>>(r, k, G, W, Q, E, flag);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

template <typename T>
ts_status launch_chol_solve(int r, int s, const T* G, const T* H, T* X, int* flag,
                            cudaStream_t st) {
  const size_t smem = sizeof(T) * ((size_t)r * r + (size_t)NWARP * r);
  TS_TRY(smem_attr((const void*)k_chol_solve<T>, smem));
  k_chol_solve<T><<<1, NT, smem, st>>>(r, s, G, H, X, flag);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

template <typename T>
ts_status launch_eig_small(int n, int R, const T* K, const T* Q, int r, T* CnT, T* Fm, T* Uout,
                           int* flag, cudaStream_t st) {
  if (n > kMaxEig) return fail(TS_ERR_SHAPE, "eigensolver: n=%d > %d", n, kMaxEig);
  const size_t smem = (size_t)n * n * (3 * sizeof(double) + 2 * sizeof(T));
  TS_TRY(smem_attr((const void*)k_eig_small<T>, smem));
  k_eig_small<T><<<1, NT, smem, st>>>(n, R, K, Q, r, CnT, Fm, Uout, flag);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

template <typename T>
ts_status launch_finalize(int s, int R, const T* V, T* A_out, T* CnT, int r, T* core, CoreMap map,
                          cudaStream_t st) {
  k_finalize<T><<<R, 256, 0, st>>>(s, R, V, A_out, CnT, r, core, map);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

#define TS_INST(T)                                                                               \
  template ts_status launch_rsvd_stage1<T>(int, int, const T*, const T*, T*, T*, int*,          \
                                           cudaStream_t);                                        \
  template ts_status launch_chol_solve<T>(int, int, const T*, const T*, T*, int*, cudaStream_t); \
  template ts_status launch_eig_small<T>(int, int, const T*, const T*, int, T*, T*, T*, int*,   \
                                         cudaStream_t);                                          \
  template ts_status launch_finalize<T>(int, int, const T*, T*, T*, int, T*, CoreMap,           \
                                        cudaStream_t);
TS_INST(float)
TS_INST(double)
#undef TS_INST

}  // namespace ts
