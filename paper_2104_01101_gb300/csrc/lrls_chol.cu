// RSVD-LRLS (Alg. 5) of one sketched subproblem on one cluster of 8 CTAs (one per SM),
// organised around short dependency chains: every CTA runs steps 1-3 and 5 on identical
// data, and the wide parts (D, K, A and the signs over column slices of H; the FP64
// products of the precision form) are split over the cluster (see "cluster exchange"
// below).  Inputs are the blocks of the augmented product [G | W | H] =
// Z^T [Z | Y Omega | Y] (G = Z^T Z, r x r SPD; W, r x k; H, r x s).
//
//   1. Symmetric elimination (G = L D L^T, L unit lower) of the augmented block [G | W],
//      held in registers by NWE warps: warp w owns the RS consecutive rows RS w ..
//      RS w + RS - 1 (whole rows: both triangles of G), lane l the 4 consecutive columns
//      4 l .. 4 l + 3 of [G | W].  As column j of G is eliminated it is replaced in place
//      by column j of N = L^{-1} (the in-place inverse), so after r steps the registers
//      hold N (strictly lower), D (diagonal) and N W.  Pivots go in groups of four, the
//      rows of one warp: their owner eliminates them among themselves and publishes the
//      four rows with their pivots' reciprocals through a double-buffered shared buffer;
//      every warp then applies the four pivots to its rows below them, each row's
//      multiplier being its own entry in the pivot's column.  One barrier per four pivots.
//      Meanwhile asynchronous copies bring this CTA's columns of H into shared memory.
//   2. B = G^{-1} = N^T D^{-1} N is never formed: C = B W = N^T (D^{-1} (N W)) and
//      E = B Q = N^T (D^{-1} (N Q)) are triangular products with k <= 16 columns.
//   3. Q = qr(C): shifted CholeskyQR3 in FP32 for FP32 data (one CTA: Gram by shuffles,
//      LDL^T in one warp's registers), Householder for FP64 data, FP64 CholeskyQR2 over
//      the cluster in the precision form.
//   4. D = E^T H (k x s; E^T H = Q^T B Z^T Y of Alg. 5) over each CTA's columns, K = D D^T
//      summed over the cluster.
//   5. K = U Lambda U^T by cyclic Jacobi on four warps (round-robin pairs; rotations of a
//      round applied as 2 x 2 block updates into a second buffer; one 128-thread barrier
//      per round); in the precision form one FP64 refinement of the eigenpairs follows.
//   6. C_(n)^T = Q U_R Sigma_R, A^(n) = D^T U_R Sigma_R^{-1}, canonical column signs, core.
#include <cooperative_groups.h>

#include "dense_la.cuh"

namespace cg = cooperative_groups;

namespace ts {

namespace {
constexpr int kCT = 512;  // threads of the block
constexpr int kCW = kCT / 32;
constexpr int kCK = 16;    // widest RSVD sketch (k) and Jacobi order
constexpr int kCKs = 17;   // row stride of the k x k Jacobi buffers
constexpr int kCX = 132;   // one pivot row: 128 columns + the pivot's reciprocal at kCX - 1
constexpr int kCMax = 128; // r + k limit of the elimination tile
constexpr int kQS = 20;    // row stride of Q and E (80 B: eight rows at one column
                           // block fall in distinct shared-memory bank groups)
constexpr unsigned kAll = 0xffffffffu;
constexpr int kNC = 8;  // CTAs of the cluster that shares one subproblem (one per SM)
// FP64 precision form: a scalar after the 16 x 17 Gram (S), and the size of the eigen
// refinement's workspace (in doubles; K's FP64 copy follows it)
constexpr int kP64Scal = 272;
constexpr int kRefineWs = 656;
}  // namespace

// Rows per warp of the elimination (all 16 warps): FP32 8 (r <= 128), FP64 4 (r <= 64,
// the register budget of 512 threads).  RS % 4 == 0 and 4 | RS keep the parity of a
// pivot and its column slot compile-time constants of the 4-pivot loop body.
template <typename T>
struct ElimShape {
  static constexpr int NWE = kCW;
  static constexpr int RS = sizeof(T) == 4 ? 8 : 4;
};

__device__ __forceinline__ void elim_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Shared-memory layout of one CTA (byte offsets).  T = data type, U = QR type; sw is the
// widest column slice of H / D / A that a CTA owns.
struct CholLayout {
  int ldn, sw;
  size_t H, D, Am, N, dinv, Y, Q, E, buf, late, C, tau, K0, K1, V, F, CnT, X, total;
  bool h_smem, d_smem, a_smem;
};

__host__ __device__ inline CholLayout chol_layout(int r, int s, int k, int R, size_t tsz,
                                                  size_t usz, bool h_smem, bool d_smem,
                                                  bool a_smem) {
  CholLayout L{};
  L.ldn = (r + 3) & ~3;
  L.sw = (s + kNC - 1) / kNC;
  L.h_smem = h_smem;
  L.d_smem = d_smem;
  L.a_smem = a_smem;
  const size_t sw = L.sw;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 15) & ~(size_t)15;
    const size_t o = off;
    off += bytes;
    return o;
  };
  // the own columns of H (r x sw) when they are copied in; D (k x sw) then overwrites
  // their first k rows and A (sw x R) follows them (row stride sw for H and D)
  if (h_smem) {
    L.H = take(tsz * (size_t)r * sw);
    L.D = L.H;
    L.Am = L.H + tsz * (size_t)k * sw;
  } else {
    L.D = take(d_smem ? tsz * (size_t)k * sw : 0);
    L.Am = take(a_smem ? tsz * sw * R : 0);
  }
  // N is dead after step 4: the FP64 eigen refinement's workspace and K's FP64 copy
  // reuse it; Y is dead during the QR: the FP64 Gram, its scalars, D^{-1/2} and the own
  // rows of C in FP64 (16 x 17 + 16 + 16 + 256 doubles)
  const size_t n_bytes = tsz * (size_t)r * L.ldn, y_bytes = tsz * (size_t)r * kCK;
  const size_t n64 = 8 * (size_t)(kRefineWs + 16 * 17), y64 = 8 * (size_t)(304 + 256);
  L.N = take(n_bytes > n64 ? n_bytes : n64);
  L.dinv = take(tsz * (size_t)((r + 3) & ~3));
  L.Y = take(y_bytes > y64 ? y_bytes : y64);
  L.Q = take(tsz * (size_t)r * kQS);
  L.E = take(tsz * (size_t)r * kQS);
  L.buf = take(tsz * 8 * kCX > 66 * 8 ? tsz * 8 * kCX : 66 * 8);
  // the QR workspace, then (after Q is formed) the Jacobi buffers and C_(n)^T
  const size_t qr = ((usz * (size_t)r * 17 + 15) & ~(size_t)15) + usz * kCK;
  const size_t kb = ((tsz * kCK * kCKs + 15) & ~(size_t)15);
  const size_t lt = 3 * kb + ((tsz * kCK * kCK + 15) & ~(size_t)15) + tsz * (size_t)r * R;
  L.late = take(qr > lt ? qr : lt);
  L.C = L.late;
  L.tau = L.late + ((usz * (size_t)r * 17 + 15) & ~(size_t)15);
  L.K0 = L.late;
  L.K1 = L.K0 + kb;
  L.V = L.K1 + kb;
  L.F = L.V + kb;
  L.CnT = L.F + ((tsz * kCK * kCK + 15) & ~(size_t)15);
  // exchange with the peers, one slot per CTA of the cluster: a 16 x 17 FP64 partial
  // (Gram or K) and the sign candidates
  L.X = take((size_t)kNC * 8 * (16 * 17 + 3 * 16));
  L.total = off;
  return L;
}

template <typename T>
struct V4;
template <>
struct V4<float> {
  __device__ static void ld(const float* p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  }
  __device__ static void st(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct V4<double> {
  __device__ static void ld(const double* p, double (&v)[4]) {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
  }
  __device__ static void st(double* p, const double (&v)[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
};

// ---------------------------------------------------------------- 1. elimination

// Reciprocal of a pivot: the hardware approximation refined by one Newton step (FP32),
// or the division (FP64).
__device__ __forceinline__ float elim_rcp(float v) {
  const float y = __fdividef(1.0f, v);
  return y * fmaf(-v, y, 2.0f);
}
__device__ __forceinline__ double elim_rcp(double v) { return 1.0 / v; }

// ---- full rows, four pivots per barrier
//
// Each warp keeps its rows of [G | W] whole (both triangles of G), so the row of a pivot
// is all in its owner warp: no column has to be gathered from the other warps.  The four
// pivot rows of group g (pivots 4g .. 4g + 3, rows of one warp) are published together,
// already eliminated among themselves by the owner; every warp then applies the four
// pivots in turn to its rows below them, a row's multiplier being its own entry in the
// pivot's column (lane g, slot b).  One barrier per four pivots.

// The owner of group g publishes its rows (slots O .. O + 3 of x, every earlier pivot
// applied), eliminated among themselves, to dst (4 x kCX; entry kCX - 1 of row b holds
// the reciprocal of pivot 4g + b).  A non-positive or non-finite pivot sets *flag and is
// replaced by 1.
template <typename T, int RS, int O>
__device__ __forceinline__ void elim_publish_group(const T (&x)[RS][4], int g, int r, T* dst,
                                                   int* flag) {
  const int lane = threadIdx.x & 31;
  T y[4][4];
#pragma unroll
  for (int b = 0; b < 4; ++b)
#pragma unroll
    for (int u = 0; u < 4; ++u) y[b][u] = x[O + b][u];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    if (4 * g + b >= r) break;
    const T d = __shfl_sync(kAll, y[b][b], g);
    const bool bad = !(d > (T)0) || !isfinite(d);
    if (bad && lane == 0 && flag) atomicExch(flag, 1);
    const T inv = elim_rcp(bad ? (T)1 : d);
    V4<T>::st(dst + b * kCX + 4 * lane, y[b]);
    if (lane == 0) dst[b * kCX + kCX - 1] = inv;
#pragma unroll
    for (int b2 = b + 1; b2 < 4; ++b2) {
      const T mm = __shfl_sync(kAll, y[b2][b], g) * inv;
#pragma unroll
      for (int u = 0; u < 4; ++u) y[b2][u] = fma(-mm, y[b][u], y[b2][u]);
      if (lane == g) y[b2][b] = -mm;  // column 4g + b of the row becomes column of N
    }
  }
}

// Group g's pivots applied to every row below them (GODD = g & 1: where the next group's
// rows sit in their owner warp), then the next group's rows published.
template <typename T, int NWE, int RS, int GODD>
__device__ __forceinline__ void elim_group_step(T (&x)[RS][4], int g, int r, T* buf, int* flag) {
  constexpr int ON = RS == 4 ? 0 : (GODD ? 0 : 4);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int rb0 = RS * w, p0 = 4 * g;
  const T* cur = buf + (g & 1) * 4 * kCX;
  T* nxt = buf + ((g & 1) ^ 1) * 4 * kCX;
  if (rb0 > p0 + 3) {  // every row of this warp is below the group: no predicates
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      if (p0 + b >= r) break;
      const T inv = cur[b * kCX + kCX - 1];
      T v[4];
      V4<T>::ld(cur + b * kCX + 4 * lane, v);
      const bool fix = lane == g;
#pragma unroll
      for (int t = 0; t < RS; ++t) {
        const T mm = __shfl_sync(kAll, x[t][b], g) * inv;
#pragma unroll
        for (int u = 0; u < 4; ++u) x[t][u] = fma(-mm, v[u], x[t][u]);
        if (fix) x[t][b] = -mm;  // column p of G becomes column p of N
      }
    }
  } else if (rb0 + RS - 1 > p0) {  // the warp that holds the group: rows below a pivot only
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int p = p0 + b;
      if (p >= r) break;
      const T inv = cur[b * kCX + kCX - 1];
      T v[4];
      V4<T>::ld(cur + b * kCX + 4 * lane, v);
#pragma unroll
      for (int t = 0; t < RS; ++t) {
        const bool act = rb0 + t > p;
        const T mm = __shfl_sync(kAll, x[t][b], g) * inv;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const T nv = fma(-mm, v[u], x[t][u]);
          x[t][u] = act ? nv : x[t][u];
        }
        if (act && lane == g) x[t][b] = -mm;
      }
    }
  }
  const int gn = g + 1;
  if (4 * gn < r && w == (4 * gn) / RS) elim_publish_group<T, RS, ON>(x, gn, r, nxt, flag);
  elim_sync(NWE * 32);
}

// Symmetric elimination of [G | W] (r + k <= 128) by warps 0 .. NWE - 1 in groups of four
// pivots (above); on exit N (unit lower, r x ldn, zeros above), dinv = D^{-1} and
// Y = N W (r x 16, zero columns >= k) are in shared memory (the caller synchronises the
// block).  A non-positive or non-finite pivot sets *flag and is replaced by 1.  Tile
// slots beyond W take harmless garbage, and the dump masks the upper triangle.
template <typename T, int NWE, int RS, typename AfterLoad>
__device__ void chol_eliminate(const T* __restrict__ G, long ldg, const T* __restrict__ W,
                               long ldw, int r, int k, T* buf, T* Nm, int ldn, T* dinv, T* Y,
                               int* flag, AfterLoad after_load) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  T x[RS][4];
#pragma unroll
  for (int t = 0; t < RS; ++t) {
    const int i = RS * w + t;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = 4 * lane + u;
      T v = (T)0;
      if (i < r) {
        if (c < r) {
          v = G[(long)i * ldg + c];
        } else if (c - r < k) {
          v = W[(long)i * ldw + (c - r)];
        }
      }
      x[t][u] = v;
    }
  }
  after_load();  // issued behind the loads of the tile, which the first step waits for
  // group 0's rows from warp 0, then one step per group of four pivots
  if (w == 0) elim_publish_group<T, RS, 0>(x, 0, r, buf, flag);
  elim_sync(NWE * 32);
  for (int g = 0; 4 * g < r; g += 2) {
    elim_group_step<T, NWE, RS, 0>(x, g, r, buf, flag);
    if (4 * (g + 1) < r) elim_group_step<T, NWE, RS, 1>(x, g + 1, r, buf, flag);
  }
  // N (unit diagonal, zeros above and in the padding columns r .. ldn - 1), D^{-1}, N W:
  // a lane's four columns of N go out as one vector store
#pragma unroll
  for (int t = 0; t < RS; ++t) {
    const int i = RS * w + t;
    if (i >= r) continue;
    const int c0 = 4 * lane;
    if (c0 < ldn) {
      T o[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int c = c0 + u;
        o[u] = c < i ? x[t][u] : (c == i ? (T)1 : (T)0);
      }
      V4<T>::st(Nm + i * ldn + c0, o);
      if (lane == (i >> 2)) {  // the diagonal: slot i & 3 = t & 3 (RS is a multiple of 4)
        T d = x[t][t & 3];
        if (!(d > (T)0) || !isfinite(d)) d = (T)1;  // flagged during elimination
        dinv[i] = (T)1 / d;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = c0 + u;
      if (c >= r && c - r < kCK) Y[i * kCK + (c - r)] = (c - r < k) ? x[t][u] : (T)0;
    }
  }
  // Y columns c with r + c >= 128 are outside the tile
  for (int e = tid; e < r * kCK; e += NWE * 32) {
    const int i = e >> 4, c = e & 15;
    if (r + c >= kCMax) Y[i * kCK + c] = (T)0;
  }
}

// ---------------------------------------------------------------- 2. triangular products

// out(i, :) = post(i) * sum_a N~(i, a) * pre(a) * in(a, :) with N~ = N^T (UPPER: a >= i,
// coefficient N(a, i)) or N (lower: a <= i, coefficient N(i, a)); N has a unit diagonal
// and zeros above it, so the sums may run over whole 4-row blocks.  in/out are r x 16;
// pre/post may be null (1); ldi, ldo: their row strides.  A thread owns a 4 x 4 block of out and a quarter of the
// sum (4-row blocks x 4 column blocks x 4 quarters = 512 threads for r <= 128).
template <typename T, bool UPPER>
__device__ void tri_product(const T* Nm, int ldn, int r, const T* pre, const T* in, int ldi,
                            const T* post, T* out, int ldo) {
  const int tid = threadIdx.x, q = tid & 3, cb = (tid >> 2) & 3, ib = tid >> 4;
  const int i0 = 4 * ib;
  T acc[4][4];
#pragma unroll
  for (int e = 0; e < 4; ++e)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[e][b] = (T)0;
  if (i0 < r) {
    const int a0 = UPPER ? i0 + q : q;
    const int a1 = UPPER ? r : min(r, i0 + 4);
#pragma unroll 2
    for (int a = a0; a < a1; a += 4) {
      T cf[4], v[4];
      if (UPPER) {
        V4<T>::ld(Nm + a * ldn + i0, cf);  // N(a, i0 .. i0 + 3)
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) cf[e] = (i0 + e < r) ? Nm[(i0 + e) * ldn + a] : (T)0;
      }
      V4<T>::ld(in + a * ldi + 4 * cb, v);
      if (pre) {
        const T p = pre[a];
#pragma unroll
        for (int b = 0; b < 4; ++b) v[b] *= p;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[e][b] = fma(cf[e], v[b], acc[e][b]);
    }
  }
#pragma unroll
  for (int e = 0; e < 4; ++e)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      acc[e][b] += __shfl_xor_sync(kAll, acc[e][b], 1);
      acc[e][b] += __shfl_xor_sync(kAll, acc[e][b], 2);
    }
  if (i0 < r && q == 0) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int i = i0 + e;
      if (i < r) {
        const T sc = post ? post[i] : (T)1;
        T o[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) o[b] = acc[e][b] * sc;
        V4<T>::st(out + i * ldo + 4 * cb, o);
      }
    }
  }
}

// ---------------------------------------------------------------- 3. Householder QR

// Thin QR of A (r x k, row stride lda, type U) by Householder reflections, warp c owning
// column c.  Warp j+1 applies reflector j to its column and then forms reflector j+1
// without a barrier in between, so one block barrier per reflector.  On exit Qout
// (r x 16, row stride kQS, type T, zero columns >= k) holds the orthonormal factor.  A zero column gives
// tau = 0 (an identity reflector).
template <typename U, typename T>
__device__ void chol_householder(U* A, int lda, int r, int k, U* tau, T* Qout) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = 0; j < k; ++j) {
    if (warp == j) {
      U sq = 0;
      for (int i = j + lane; i < r; i += 32) {
        const U v = A[i * lda + j];
        sq += v * v;
      }
      sq = warp_sum(sq);
      const U ajj = A[j * lda + j];
      U tj = 0, v0 = ajj;
      if (sq > (U)0) {
        const U alpha = ajj >= (U)0 ? -sqrt(sq) : sqrt(sq);
        v0 = ajj - alpha;
        const U vn2 = sq - ajj * ajj + v0 * v0;
        tj = vn2 > (U)0 ? (U)2 / vn2 : (U)0;
      }
      __syncwarp();
      if (lane == 0) {
        A[j * lda + j] = v0;
        tau[j] = tj;
      }
    }
    __syncthreads();
    if (warp > j && warp < k) {
      const U tj = tau[j];
      U wsum = 0;
      for (int i = j + lane; i < r; i += 32) wsum += A[i * lda + j] * A[i * lda + warp];
      wsum = warp_sum(wsum) * tj;
      for (int i = j + lane; i < r; i += 32) A[i * lda + warp] -= wsum * A[i * lda + j];
      __syncwarp();
    }
  }
  __syncthreads();
  if (warp < kCK) {  // Q(:, c) = H_0 ... H_c e_c; columns >= k are zero
    const int c = warp;
    U q[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int i = lane + 32 * t;
      q[t] = (c < k && i == c) ? (U)1 : (U)0;
    }
    if (c < k) {
      for (int j = c; j >= 0; --j) {
        const U tj = tau[j];
        U wsum = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int i = lane + 32 * t;
          if (i >= j && i < r) wsum += A[i * lda + j] * q[t];
        }
        wsum = warp_sum(wsum) * tj;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int i = lane + 32 * t;
          if (i >= j && i < r) q[t] -= wsum * A[i * lda + j];
        }
      }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int i = lane + 32 * t;
      if (i < r) Qout[i * kQS + c] = (T)q[t];
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- 3b. FP32 shifted CholeskyQR3

// Q = qr(C) for FP32 data by shifted CholeskyQR3 (Fukaya, Kannan, Nakatsukasa, Yamamoto
// and Yanagisawa, SIAM J. Sci. Comput. 42 (2020)): a Cholesky-QR pass on C^T C + s I with
// s = 11 (r k + k (k + 1)) u ||C||_F^2 (u = 2^-24) leaves Q1 with a condition number the
// unshifted passes can take, and two unshifted passes follow.  Each pass is one CTA on
// its own data (no cluster exchange): the Gram by 10 warps (one 4 x 4 block of the lower
// triangle each, rows over the lanes, then a butterfly reduce-scatter of the 16 sums),
// the LDL^T in one warp's registers (no block barrier), the product by all threads.
// Alg. 5 uses Q only as a basis of range(C), so the sign of each column (positive here,
// the reflection's there) does not matter.

__device__ __forceinline__ bool cq_above(float x, float thr) {
  return __float_as_int(x) > __float_as_int(thr);  // thr >= +0: x > thr, x not a NaN
}

// S = C^T C (16 x 17, both triangles; columns >= k of C read as zero).  Warp w < 10 owns
// block (bi, bc), bi >= bc; lane l sums rows l, l + 32, l + 64, l + 96.
__device__ __forceinline__ void cq_gram(const float* C, int r, int k, float* S) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (w >= 10) return;
  const int bi = w < 1 ? 0 : w < 3 ? 1 : w < 6 ? 2 : 3;  // w = bi (bi + 1) / 2 + bc
  const int bc = w - bi * (bi + 1) / 2;
  float acc[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) acc[u] = 0.f;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const int i = lane + 32 * t;
    if (i < r) {
      float a[4], b[4];
      V4<float>::ld(C + i * kQS + 4 * bi, a);
      V4<float>::ld(C + i * kQS + 4 * bc, b);
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        a[x] = 4 * bi + x < k ? a[x] : 0.f;
        b[x] = 4 * bc + x < k ? b[x] : 0.f;
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[4 * x + y] = fmaf(a[x], b[y], acc[4 * x + y]);
    }
  }
  // reduce-scatter: afterwards lanes 2v and 2v + 1 hold the warp's total of sum v
#pragma unroll
  for (int h = 8, o = 16; h >= 1; h >>= 1, o >>= 1) {
    const bool up = lane & o;
#pragma unroll
    for (int u = 0; u < h; ++u) {
      const float send = up ? acc[u] : acc[u + h];
      const float keep = up ? acc[u + h] : acc[u];
      acc[u] = keep + __shfl_xor_sync(kAll, send, o);
    }
  }
  acc[0] += __shfl_xor_sync(kAll, acc[0], 1);
  if ((lane & 1) == 0) {
    const int x = lane >> 3, y = (lane >> 1) & 3;
    S[(4 * bi + x) * kCKs + 4 * bc + y] = acc[0];
    S[(4 * bc + y) * kCKs + 4 * bi + x] = acc[0];
  }
}

// The factor of one pass in warp 0: S + shift I = N^{-1} D N^{-T}, written as Nt = N^T
// (16 x 16: Nt[a][c] = N(c, a), unit diagonal, zeros below) and dsq = D^{-1/2} (a pivot
// not above thr drops its direction: dsq = 0).  Lane l holds row l / 2, columns
// 8 (l % 2) .. + 7; pivot j's row, the lane's own entry in column j and the pivot come
// by shuffles.  The pivot loop is unrolled by 8 (the slot index a constant, one copy of
// the code for both halves) and has no branch, so a step's trailing updates overlap the
// next step's shuffles.  mode 0: shifted first pass; 1: full LDL^T; 2: first order when
// S is within 2^-12 of I (N = I - strictly_lower(S - I), D^{-1/2} = I - diag(S - I) / 2,
// error second order), else full.
__device__ __forceinline__ void cq_factor(const float* S, int r, int k, int mode, float* Nt,
                                          float* dsq) {
  const int lane = threadIdx.x & 31, i = lane >> 1, h = lane & 1;
  float v[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int c = 8 * h + u;
    v[u] = (i < k && c < k) ? S[i * kCKs + c] : 0.f;
  }
  float tr = lane < k ? S[lane * kCKs + lane] : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(kAll, tr, o);
  bool first_order = false;
  if (mode == 2) {
    bool off = false;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = 8 * h + u;
      if (i < k && c < k) off |= !(fabsf(v[u] - (c == i ? 1.f : 0.f)) <= 0x1.0p-12f);
    }
    first_order = !__any_sync(kAll, off);
  }
  float dq = 0.f;
  if (first_order) {
    if (lane < k) dq = 1.5f - 0.5f * S[lane * kCKs + lane];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = 8 * h + u < i ? -v[u] : 0.f;
  } else {
    float thr = k > 0 ? 0x1.0p-40f * tr / (float)k : 0.f;
    if (mode == 0) {  // the shift, on the diagonal
      thr = 0.f;
      const float sh = 11.f * (float)(r * k + k * (k + 1)) * 0x1.0p-24f * tr;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (8 * h + u == i && i < k) v[u] += sh;
    }
#pragma unroll 1
    for (int q = 0; q < 2; ++q) {  // pivots 8 q .. 8 q + 7: column 8 q + t is slot t of half q
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int j = 8 * q + t;
        const float d = __shfl_sync(kAll, v[t], 17 * q + 2 * t);
        const float sij = __shfl_sync(kAll, v[t], 2 * i + q);
        float rowj[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) rowj[u] = __shfl_sync(kAll, v[u], 16 * q + 2 * t + h);
        const float dinv = cq_above(d, thr) ? elim_rcp(d) : 0.f;
        dq = lane == j ? dinv : dq;
        const float m = i > j ? sij * dinv : 0.f;  // rows up to j: unchanged
#pragma unroll
        for (int u = 0; u < 8; ++u)
          v[u] = (u == t && h == q && i > j) ? -m : fmaf(-m, rowj[u], v[u]);
      }
    }
    dq = sqrtf(dq);
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int c = 8 * h + u;
    Nt[c * kCK + i] = c < i ? v[u] : (c == i ? 1.f : 0.f);
  }
  if (lane < kCK) dsq[lane] = lane < k ? dq : 0.f;
}

// One pass: Qout = C N^T D^{-1/2} (r x 16, zero columns >= k; both with row stride kQS);
// Qout must not be C.  ws:
// 16 x 17 + 16 x 16 + 16 floats, 16-byte aligned.
__device__ __forceinline__ void cq_pass(const float* C, float* Qout, int r, int k, int mode,
                                        float* ws) {
  float* S = ws;
  float* Nt = ws + kCK * kCKs;
  float* dsq = Nt + kCK * kCK;
  cq_gram(C, r, k, S);
  __syncthreads();
  if (threadIdx.x < 32) cq_factor(S, r, k, mode, Nt, dsq);
  __syncthreads();
  const int i = threadIdx.x >> 2, cg = threadIdx.x & 3;
  if (i < r) {
    float crow[4][4], acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      V4<float>::ld(C + i * kQS + 4 * b, crow[b]);
#pragma unroll
      for (int x = 0; x < 4; ++x) crow[b][x] = 4 * b + x < k ? crow[b][x] : 0.f;
    }
#pragma unroll
    for (int a = 0; a < kCK; ++a) {
      float nv[4];
      V4<float>::ld(Nt + a * kCK + 4 * cg, nv);  // N(4 cg .. 4 cg + 3, a)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[e] = fmaf(crow[a >> 2][a & 3], nv[e], acc[e]);
    }
    float dv[4], o[4];
    V4<float>::ld(dsq + 4 * cg, dv);
#pragma unroll
    for (int e = 0; e < 4; ++e) o[e] = 4 * cg + e < k ? acc[e] * dv[e] : 0.f;
    V4<float>::st(Qout + i * kQS + 4 * cg, o);
  }
  __syncthreads();
}

// Shifted CholeskyQR3: C (r x 16, FP32, row stride kQS) -> Q; B is scratch of the same shape
// (C may be B).
// The passes run as one loop, so their code is fetched once.
__device__ void cq3_f32(const float* C, float* B, float* Q, int r, int k, float* ws) {
#pragma unroll 1
  for (int p = 0; p < 3; ++p) cq_pass(p == 0 ? C : (p == 1 ? Q : B), p == 1 ? B : Q, r, k, p, ws);
}

// ---------------------------------------------------------------- 5. Jacobi on four warps

template <typename T>
__host__ __device__ constexpr T cj_tol() {
  return sizeof(T) == 4 ? (T)4.8e-7 : (T)8.9e-16;  // 8 unit roundoffs
}
template <typename T>
__host__ __device__ constexpr T cj_floor() {
  return sizeof(T) == 4 ? (T)1.2e-7 : (T)2.2e-16;  // 2 unit roundoffs
}

// 1 / sqrt(x) to working precision (one Newton step on the hardware approximation)
__device__ __forceinline__ float cj_rsqrt(float x) {
  const float y = rsqrtf(x);
  return y * fmaf(-0.5f * x * y, y, 1.5f);
}
__device__ __forceinline__ double cj_rsqrt(double x) { return 1.0 / sqrt(x); }

// Pair a (0..7) of round t (0..14) of the round-robin schedule on 16 indices.
__device__ __forceinline__ void cj_pair(int t, int a, int& p, int& q) {
  int x = t + a, y = t - a + 15;
  x = x >= 15 ? x - 15 : x;
  y = y >= 15 ? y - 15 : y;
  if (a == 0) {
    x = t;
    y = 15;
  }
  p = min(x, y);
  q = max(x, y);
}

// Rotation J = [[c, s], [-s, c]] on (p, q) with (J^T A J)(p, q) = 0, from the half-angle
// form: with x = a_qq - a_pp, y = 2 a_pq, cos^2(phi) = (1 + |x| / sqrt(x^2 + y^2)) / 2
// and sin(phi) = sign(x) y / (2 sqrt(x^2 + y^2) cos(phi)) (tan(phi) = t, the root of
// t^2 + 2 theta t - 1 = 0 of smaller magnitude, theta = x / y).  Both reciprocal square
// roots are refined to working precision, so c^2 + s^2 = 1 to rounding.
template <typename T>
__device__ __forceinline__ void cj_rotation(T app, T aqq, T apq, bool rot, T& c, T& s) {
  const T x = aqq - app, y = 2 * apq;
  const T h = fma(x, x, y * y);
  const T ih = cj_rsqrt(rot ? h : (T)1);
  const T c2 = fma((T)0.5 * fabs(x), ih, (T)0.5);
  const T rc = cj_rsqrt(c2);
  c = rot ? c2 * rc : (T)1;
  s = rot ? (x >= (T)0 ? y : -y) * ((T)0.5 * ih * rc) : (T)0;
}

// The same rotation for a small angle, |a_pq| <= g |x| (g = 2^-7 in FP32, 2^-14 in FP64):
// t = tan(phi) = (a_pq / x) (1 - (a_pq / x)^2) (relative error O((a_pq / x)^4)),
// c = 1 - t^2 / 2 and s = t c, for which c^2 + s^2 - 1 = -3 t^4 / 4 + O(t^6), below
// 3 g^4 / 4 (2^-30 in FP32, 2^-58 in FP64): one reciprocal instead of two refined
// reciprocal square roots.
template <typename T>
__host__ __device__ constexpr T cj_small() {
  return sizeof(T) == 4 ? (T)128 : (T)16384;  // 1 / g
}
template <typename T>
__device__ __forceinline__ void cj_rotation_small(T app, T aqq, T apq, bool rot, T& c, T& s) {
  const T u = apq * elim_rcp(rot ? aqq - app : (T)1);
  const T t = u * fma(-u, u, (T)1);
  c = rot ? fma((T)-0.5 * t, t, (T)1) : (T)1;
  s = rot ? t * c : (T)0;
}


// Symmetric eigen-decomposition of K (16 x 16, row stride kCKs, zero-padded beyond the
// order) by cyclic Jacobi on warps 0 .. kJW - 1 (the caller's other threads skip it):
// K <- V^T K V, V (start: identity) holds the eigenvectors.  A pair rotates when |a_pq|
// exceeds both tol sqrt(|a_pp a_qq|) and floor max_i |a_ii|; a sweep whose largest |sin|
// is at most sqrt(tol) ends the loop (quadratic convergence: the next sweep's angles
// would be ~tol).  Round t rotates the 8 disjoint pairs of the round-robin schedule.  In
// every warp lane L forms the rotation of pair a = L & 7 (all warps the same values);
// warps 0 and 1 update the 2 x 2 block (a, b) of A into B for the column pair
// b = 2 (L >> 3) + w (its rotation by shuffle from lane b), warps 2 and 3 rotate
// columns p, q of V in rows 4 (L >> 3) + 2 (w - 2) and the next.  Spreading the round
// over four warps cuts each warp's instructions per round (the round is a latency chain
// of loads, two refined reciprocal square roots, a shuffle and stores); one 128-thread
// barrier per round.  Returns the buffer holding the diagonalised matrix.
constexpr int kJW = 4;
__device__ __forceinline__ void cj_sync() { asm volatile("bar.sync 3, 128;" ::: "memory"); }

template <typename T>
__device__ T* cj_jacobi(T* K, T* K2, T* V, int max_sweeps) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int e = tid; e < kCK * kCK; e += 32 * kJW) {
    const int i = e >> 4, j = e & 15;
    V[i * kCKs + j] = i == j ? (T)1 : (T)0;
  }
  T dmax = 0;
  if (lane < 16) dmax = fabs(K[lane * kCKs + lane]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(kAll, dmax, o));
  const T tol = cj_tol<T>(), tol2 = tol * tol, floor_abs = cj_floor<T>() * dmax;
  const float stop_s = sqrtf((float)tol);
  cj_sync();
  T* A = K;
  T* B = K2;
  const int a = lane & 7, g = lane >> 3;
  const bool blk = w < 2;
  const int cb = 2 * g + (w & 1);   // the block's column pair (warps 0, 1)
  const int vr = 4 * g + 2 * (w & 1);  // the first of the two V rows (warps 2, 3)
  int p, q, pb, qb;  // this round's pairs; the next round's are formed during the round
  cj_pair(0, a, p, q);
  cj_pair(0, cb, pb, qb);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    bool any = false;
    float smax = 0.f;
    for (int t = 0; t < 15; ++t) {
      const T app = A[p * kCKs + p], aqq = A[q * kCKs + q], apq = A[p * kCKs + q];
      T x0, x1, x2, x3;
      if (blk) {
        x0 = A[p * kCKs + pb];
        x1 = A[p * kCKs + qb];
        x2 = A[q * kCKs + pb];
        x3 = A[q * kCKs + qb];
      } else {
        x0 = V[vr * kCKs + p];
        x1 = V[vr * kCKs + q];
        x2 = V[(vr + 1) * kCKs + p];
        x3 = V[(vr + 1) * kCKs + q];
      }
      int np, nq, npb, nqb;
      cj_pair(t == 14 ? 0 : t + 1, a, np, nq);
      cj_pair(t == 14 ? 0 : t + 1, cb, npb, nqb);
      T c, s;
      const bool rot = apq * apq > tol2 * fabs(app * aqq) && fabs(apq) > floor_abs;
      // every rotating pair of the round at a small angle (the same in all warps): the
      // one-reciprocal form
      if (__all_sync(kAll, !rot || fabs(apq) * cj_small<T>() <= fabs(aqq - app)))
        cj_rotation_small<T>(app, aqq, apq, rot, c, s);
      else
        cj_rotation<T>(app, aqq, apq, rot, c, s);
      if (rot && lane < 8) {
        any = true;
        smax = fmaxf(smax, (float)fabs(s));
      }
      const T cj = __shfl_sync(kAll, c, cb), sj = __shfl_sync(kAll, s, cb);
      if (blk) {  // J_a^T X J_b
        const T t00 = c * x0 - s * x2, t01 = c * x1 - s * x3;
        const T t10 = s * x0 + c * x2, t11 = s * x1 + c * x3;
        B[p * kCKs + pb] = cj * t00 - sj * t01;
        B[p * kCKs + qb] = sj * t00 + cj * t01;
        B[q * kCKs + pb] = cj * t10 - sj * t11;
        B[q * kCKs + qb] = sj * t10 + cj * t11;
      } else {  // V J_a
        V[vr * kCKs + p] = c * x0 - s * x1;
        V[vr * kCKs + q] = s * x0 + c * x1;
        V[(vr + 1) * kCKs + p] = c * x2 - s * x3;
        V[(vr + 1) * kCKs + q] = s * x2 + c * x3;
      }
      cj_sync();
      T* tmp = A;
      A = B;
      B = tmp;
      p = np;
      q = nq;
      pb = npb;
      qb = nqb;
    }
    any = __any_sync(kAll, any);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) smax = fmaxf(smax, __shfl_xor_sync(kAll, smax, o));
    if (!any || smax <= stop_s) break;
  }
  return A;
}

// ---------------------------------------------------------------- cluster exchange

// The CTAs of the cluster share one subproblem: every CTA repeats the short serial chains
// (elimination, triangular products, FP32 QR, Jacobi) on identical data, so they
// hold identical results, and each owns a slice of the work that is wide rather than
// deep: columns [j0, j1) of H, D and A, rows [i0, i1) of C for the FP64 products and two
// columns of the 16 x 16 eigen refinement.  Partial results are pushed: a CTA stores its
// part into its own slot (or rows) of every CTA's buffer through distributed shared
// memory, a cluster barrier (release / acquire) makes the stores visible, and every read
// is then local (sums always in rank order, so every CTA gets the same bits).
template <typename P>
__device__ __forceinline__ P* cl_peer(P* p, int rank) {
  return cg::this_cluster().map_shared_rank(p, rank);
}
__device__ __forceinline__ void cl_sync() { cg::this_cluster().sync(); }

// ---------------------------------------------------------------- FP64 precision form
//
// On this part an FP64 warp instruction occupies its SM sub-partition's FP64 unit for
// about 64 cycles (conversions to and from FP32 included), so the FP64 code keeps the
// instruction count low: operands converted once, FP64 work split over the cluster and,
// within a CTA, over warps on all four sub-partitions.

// FP64 reciprocal: the approximate FP64 reciprocal y (relative error e = 1 - x y below
// 2^-19; 2^-19.95 measured over 2^20 inputs on GB300) corrected by the series
// 1 / x = y / (1 - e) = y (1 + e + e^2 + ...) to second order, y + y (e + e^2): the
// truncation error is e^3 < 2^-57, one FP64 operation fewer than two Newton steps.
__device__ __forceinline__ double p64_rcp(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

// x > thr for thr >= +0, compared on the bit patterns (integer unit): a negative x is
// not above; neither is a NaN with its sign bit set (a NaN input reaches the outputs
// through the other entries of its row and column anyway).
__device__ __forceinline__ bool p64_above(double x, double thr) {
  return __double_as_longlong(x) > __double_as_longlong(thr);
}

__device__ __forceinline__ void p64_sync() { asm volatile("bar.sync 2, 256;" ::: "memory"); }

// LDL^T of a symmetric k x k FP64 matrix (k <= 16) held one entry per thread by threads
// 0..255 (thread t: row t / 16, column t % 16; entries outside k x k are zero), with
// L^{-1} = N formed in place.  On return v holds N(i, c) for c < i; the diagonal thread
// returns D(i)^{-1} (0 for a pivot not above thr: the direction is dropped), the others
// return 0.  Pivot j's row, column and reciprocal go out through a double-buffered shared
// row (pub: 2 x 33 doubles); the owner of pivot j + 1 publishes its reciprocal as soon as
// its own update is done: one barrier (256 threads) per pivot.  A warp with no row below
// the pivot only waits, and each entry takes one FP64 multiply and one fused multiply-add
// per pivot.
__device__ double p64_ldl(double& v, int k, double thr, double* pub) {
  const int t = threadIdx.x, i = t >> 4, c = t & 15, wp = t >> 5;
  double dinv = 0.0;
  if (i == 0) pub[c] = v;
  if (c == 0) pub[16 + i] = v;
  if (t == 0) pub[32] = p64_above(v, thr) ? p64_rcp(v) : 0.0;
  p64_sync();
  for (int j = 0; j < k; ++j) {
    const double* cur = pub + (j & 1) * 33;
    double* nxt = pub + ((j & 1) ^ 1) * 33;
    if (i == j && c == j) dinv = cur[32];
    if (2 * wp + 1 > j && 2 * wp < k && i > j && i < k) {
      const double m = cur[16 + i] * cur[32];
      const bool piv = c == j;  // column j of S becomes column j of N: -m
      v = fma(-m, piv ? 1.0 : cur[c], piv ? 0.0 : v);  // c < j: N's row; c > j: Schur
    }
    const int jn = j + 1;
    if (jn < k) {
      if (i == jn) nxt[c] = v;
      if (c == jn) nxt[16 + i] = v;
      if (i == jn && c == jn) nxt[32] = p64_above(v, thr) ? p64_rcp(v) : 0.0;
    }
    p64_sync();
  }
  return dinv;
}

// One FP64 Cholesky-QR pass over the cluster: Qout = C N^T D^{-1/2} with
// C^T C = N^{-1} D N^{-T}.  C (r x 16, row stride kQS, type T, columns >= k ignored) is identical in every
// CTA; this CTA owns rows [i0, i1).  A pivot not above 2^-40 ||C||_F^2 / k drops its
// direction (a zero column of Qout): below that level the Gram's own rounding decides
// the pivot, and C, computed from FP32 data, holds nothing there.  In the second pass
// (`second`) of CholeskyQR2 the Gram is usually within 2^-20 of the identity (the first
// pass leaves Q1 orthonormal to u kappa(C)^2 plus the data type's rounding); its factor
// is then taken to first order, N = I - strictly_lower(S - I), D^{-1/2} = I - diag(S - I)
// / 2, whose error is second order (below 2^-40); otherwise the full LDL^T runs again.
// On return every CTA holds all of Qout (zero columns >= k; Qout may be C).  S: 16 x 17
// FP64 and a scalar after it (kP64Scal); dsq: 16; Cd: 16 x 16 FP64 (own rows); Xg: kNC
// slots of 16 x 17 FP64 (the peers store theirs here); pub: 66 FP64.
template <typename T>
__device__ void p64_cholqr_pass(const T* C, T* Qout, int r, int k, int i0, int i1, bool second,
                                double* S, double* dsq, double* Cd, double* Xg, double* pub) {
  const int tid = threadIdx.x, cr = (int)cg::this_cluster().block_rank();
  const int nr = i1 - i0;
  for (int e = tid; e < nr * kCK; e += kCT) {
    const int ii = e >> 4, c = e & 15;
    Cd[e] = c < k ? (double)C[(i0 + ii) * kQS + c] : 0.0;
  }
  __syncthreads();
  // Gram of the own rows (2 threads per entry of the lower triangle: FP64 instructions
  // occupy the pipe for ~64 cycles per warp, so fewer warps with longer sums), to the peers
  const int npair = k * (k + 1) / 2;
  for (int e = tid; e < 2 * ((npair + 255) / 256) * 256; e += kCT) {
    const int pr = e >> 1, part = e & 1;
    double acc = 0;
    int a = 0, b = 0;
    if (pr < npair) {  // pair index -> (a, b), a <= b
      int rem = pr;
      while (rem >= k - a) {
        rem -= k - a;
        ++a;
      }
      b = a + rem;
      for (int ii = part; ii < nr; ii += 2) acc = fma(Cd[ii * kCK + a], Cd[ii * kCK + b], acc);
    }
    acc += __shfl_xor_sync(kAll, acc, 1);
    if (pr < npair && part == 0) {
#pragma unroll
      for (int q = 0; q < kNC; ++q) cl_peer(Xg, q)[cr * 272 + b * 17 + a] = acc;
    }
  }
  cl_sync();
  const int i = tid >> 4, c = tid & 15;
  const bool ent = tid < 256 && c <= i && i < k;
  if (ent) {
    double sum = 0;
#pragma unroll
    for (int q = 0; q < kNC; ++q) sum += Xg[q * 272 + i * 17 + c];
    S[i * 17 + c] = sum;
    S[c * 17 + i] = sum;
  }
  __syncthreads();
  const bool near_identity =
      second && !__syncthreads_or(ent && fabs(S[i * 17 + c] - (i == c ? 1.0 : 0.0)) > 0x1.0p-20);
  if (near_identity) {
    if (ent) {
      const double v = S[i * 17 + c];
      if (c < i) S[i * 17 + c] = -v;
      if (c == i) {
        dsq[i] = 1.0 - 0.5 * (v - 1.0);
        S[i * 17 + i] = 1.0;
      }
    }
  } else {
    if (tid < 32) {  // the drop threshold, once
      double tr = tid < k ? S[tid * 17 + tid] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(kAll, tr, o);
      if (tid == 0) S[kP64Scal] = 0x1.0p-40 * tr / k;
    }
    __syncthreads();
    if (tid < 256) {
      const double thr = S[kP64Scal];
      double v = (i < k && c < k) ? S[i * 17 + c] : 0.0;
      const double dinv = p64_ldl(v, k, thr, pub);
      if (i < k && c < k) S[i * 17 + c] = c < i ? v : (c == i ? 1.0 : 0.0);
      if (i < k && c == i) dsq[i] = dinv;
    }
    __syncthreads();
    if (tid < k) dsq[tid] = sqrt(dsq[tid]);
  }
  __syncthreads();
  // own rows of Qout: Qout(i, c) = dsq_c sum_{a <= c} C(i, a) N(c, a)
  for (int e = tid; e < nr * kCK; e += kCT) {
    const int ii = e >> 4, cc = e & 15;
    double acc = 0;
    if (cc < k)
      for (int a = 0; a <= cc; ++a) acc = fma(Cd[ii * kCK + a], S[cc * 17 + a], acc);
    const T qv = cc < k ? (T)(acc * dsq[cc]) : (T)0;
#pragma unroll
    for (int q = 0; q < kNC; ++q) cl_peer(Qout, q)[(i0 + ii) * kQS + cc] = qv;
  }
  cl_sync();
}

// One FP64 refinement of the eigen-decomposition K ~ X diag(lambda) X^T from the FP32
// Jacobi (iterative refinement for symmetric eigenproblems, Ogita & Aishima 2018):
// R = I - X^T X, S = X^T K X, lambda_j = S_jj / (1 - R_jj), and for a != j
// E_aj = (S_aj + mu_j R_aj) / (mu_j - mu_a) when the eigenvalues are apart
// (|mu_j - mu_a| > 1e-5 max |mu|), else R_aj / 2 (a cluster: only its subspace is
// determined); E_jj = R_jj / 2; X <- X + X E.  mu are the Jacobi's eigenvalues: they
// enter E only through the gaps and through mu_j R_aj with R_aj itself of the order of the
// Jacobi's error, so their error reaches X at second order.  This CTA computes columns
// 2 cr, 2 cr + 1 of E and of X + X E (4 threads per entry) and lambda for them, stores
// them into every CTA's Xn and lam, and after one cluster barrier converts the whole of
// Xn and lam.  Kd: K in FP64 (16 x 17); X (16 x 17, T, columns are eigenvectors) is
// overwritten, and so is the diagonal of Kf (T; the Jacobi's eigenvalues on entry).  ws:
// kRefineWs FP64 (Xn and lam receive the peers' columns).
template <typename T>
__device__ void p64_eig_refine(const double* Kd, T* X, T* Kf, double* ws) {
  const int tid = threadIdx.x, cr = (int)cg::this_cluster().block_rank();
  double* Xd = ws;        // X in FP64, 16 x 17
  double* Yc = ws + 272;  // y_j = K x_j for the own j, 2 x 16
  double* Ec = ws + 304;  // own columns of E, 16 x 2
  double* mu = ws + 336;  // Jacobi eigenvalues (16) and max |mu| (at 16)
  double* Xn = ws + 360;  // X + X E: own columns written here, read by the peers
  double* lam = ws + 632; // refined lambda: own entries written here, read by the peers
  if (tid < 256) Xd[(tid >> 4) * 17 + (tid & 15)] = (double)X[(tid >> 4) * kCKs + (tid & 15)];
  if (tid >= 256 && tid < 288) {  // warp 8
    const int l = tid & 15;
    const double m = (double)Kf[l * kCKs + l];
    double mx = fabs(m);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(kAll, mx, o));
    if (tid < 272) mu[l] = m;
    if (tid == 256) mu[16] = mx;
  }
  __syncthreads();
  // thread: entry (a, j) of an own column j, quarter q of its 16-term sums
  const int q = tid & 3, a = (tid >> 2) & 15, j = 2 * cr + ((tid >> 6) & 1);
  const bool act = tid < 128;
  if (act) {  // y_j(a) = sum_b K(a, b) X(b, j)
    double acc = 0;
#pragma unroll
    for (int b = 4 * q; b < 4 * q + 4; ++b) acc = fma(Kd[a * 17 + b], Xd[b * 17 + j], acc);
    acc += __shfl_xor_sync(kAll, acc, 1);
    acc += __shfl_xor_sync(kAll, acc, 2);
    if (q == 0) Yc[(j & 1) * 16 + a] = acc;
  }
  __syncthreads();
  if (act) {  // S_aj = x_a . y_j, R_aj = delta_aj - x_a . x_j, then E_aj
    double sv = 0, xv = 0;
#pragma unroll
    for (int b = 4 * q; b < 4 * q + 4; ++b) {
      sv = fma(Xd[b * 17 + a], Yc[(j & 1) * 16 + b], sv);
      xv = fma(Xd[b * 17 + a], Xd[b * 17 + j], xv);
    }
    sv += __shfl_xor_sync(kAll, sv, 1);
    sv += __shfl_xor_sync(kAll, sv, 2);
    xv += __shfl_xor_sync(kAll, xv, 1);
    xv += __shfl_xor_sync(kAll, xv, 2);
    if (q == 0) {
      const double rv = (a == j ? 1.0 : 0.0) - xv;
      double e;
      if (a == j) {
        e = 0.5 * rv;
        const double lj = sv / (1.0 - rv);
#pragma unroll
        for (int p = 0; p < kNC; ++p) cl_peer(lam, p)[j] = lj;
      } else {
        const double gap = mu[j] - mu[a];
        e = fabs(gap) > 1e-5 * mu[16] ? (sv + mu[j] * rv) / gap : 0.5 * rv;
      }
      Ec[a * 2 + (j & 1)] = e;
    }
  }
  __syncthreads();
  if (act) {  // own columns of X + X E
    double acc = 0;
#pragma unroll
    for (int b = 4 * q; b < 4 * q + 4; ++b) acc = fma(Xd[a * 17 + b], Ec[b * 2 + (j & 1)], acc);
    acc += __shfl_xor_sync(kAll, acc, 1);
    acc += __shfl_xor_sync(kAll, acc, 2);
    if (q == 0) {
      const double xn = Xd[a * 17 + j] + acc;
#pragma unroll
      for (int p = 0; p < kNC; ++p) cl_peer(Xn, p)[a * 17 + j] = xn;
    }
  }
  cl_sync();
  if (tid < 256) X[(tid >> 4) * kCKs + (tid & 15)] = (T)Xn[(tid >> 4) * 17 + (tid & 15)];
  if (tid >= 256 && tid < 256 + kCK) Kf[(tid - 256) * kCKs + (tid - 256)] = (T)lam[tid - 256];
  __syncthreads();
}

// ---------------------------------------------------------------- the kernel

template <typename T, typename U, bool P64>
__device__ __forceinline__ void lrls_chol_body(const FusedArgs<T>& a, bool h_smem) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int order[kCK];
  __shared__ T sgn[kCK];
  __shared__ T* Kfin;
  constexpr int NWE = ElimShape<T>::NWE, RS = ElimShape<T>::RS;
  const int r = a.r, s = a.s, k = a.k, R = a.R;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cr = (int)cg::this_cluster().block_rank();
  const CholLayout L =
      chol_layout(r, s, k, R, sizeof(T), sizeof(U), h_smem, a.m_smem, a.m_smem);
  // this CTA's columns of H / D / A and rows of C
  const int j0 = (int)((long)s * cr / kNC), w = (int)((long)s * (cr + 1) / kNC) - j0;
  const int i0 = r * cr / kNC, i1 = r * (cr + 1) / kNC;
  const int sw = L.sw;
  T* Hs = reinterpret_cast<T*>(smem_raw + L.H);
  T* Nm = reinterpret_cast<T*>(smem_raw + L.N);
  T* dinv = reinterpret_cast<T*>(smem_raw + L.dinv);
  T* Y = reinterpret_cast<T*>(smem_raw + L.Y);
  U* Cq = reinterpret_cast<U*>(smem_raw + L.C);
  U* tau = reinterpret_cast<U*>(smem_raw + L.tau);
  T* Q = reinterpret_cast<T*>(smem_raw + L.Q);
  T* E = reinterpret_cast<T*>(smem_raw + L.E);
  T* buf = reinterpret_cast<T*>(smem_raw + L.buf);
  T* K0 = reinterpret_cast<T*>(smem_raw + L.K0);
  T* K1 = reinterpret_cast<T*>(smem_raw + L.K1);
  T* V = reinterpret_cast<T*>(smem_raw + L.V);
  T* F = reinterpret_cast<T*>(smem_raw + L.F);
  T* CnTs = reinterpret_cast<T*>(smem_raw + L.CnT);
  // exchange slots (one per CTA): Gram / K partials, then the sign candidates
  double* Xg = reinterpret_cast<double*>(smem_raw + L.X);
  T* Xbest = reinterpret_cast<T*>(smem_raw + L.X + (size_t)kNC * 16 * 17 * 8);
  T* Xval = Xbest + kNC * kCK;
  int* Xidx = reinterpret_cast<int*>(Xval + kNC * kCK);
  // D (k x w) and A (w x R) of the own columns: in shared memory (row stride sw for D)
  // or in the caller's buffers (row stride s for D; A's rows j0 .. j0 + w - 1)
  const bool d_sm = h_smem || L.d_smem, a_sm = h_smem || L.a_smem;
  T* D = d_sm ? reinterpret_cast<T*>(smem_raw + L.D) : a.Mbuf + j0;
  const long ldd = d_sm ? sw : s;
  T* Am = a_sm ? reinterpret_cast<T*>(smem_raw + L.Am) : a.A_out + (long)j0 * R;
  const T* Hsrc = h_smem ? Hs : a.H + j0;
  const long ldh = h_smem ? sw : a.ldh;

  // 1. G = L D L^T with N = L^{-1} and N W, while the own columns of H stream into
  //    shared memory by asynchronous copies issued once the tile's loads are out
  //    (waited for before step 5)
  auto copy_h = [&]() {
    if (!h_smem) return;
    for (int e = tid; e < r * w; e += kCT) {
      const int i = e / w, jj = e - i * w;
      const T* src = a.H + (long)i * a.ldh + j0 + jj;
      const unsigned d = (unsigned)__cvta_generic_to_shared(Hs + (long)i * sw + jj);
      if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
      else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
    }
  };
  chol_eliminate<T, NWE, RS>(a.G, a.ldg, a.W, a.ldw, r, k, buf, Nm, L.ldn, dinv, Y, a.flag,
                             copy_h);
  __syncthreads();
  // 2. C = N^T D^{-1} (N W)
  if constexpr (P64 || sizeof(T) == 4) {  // staged in E (free until step 4)
    tri_product<T, true>(Nm, L.ldn, r, dinv, Y, kCK, nullptr, E, kQS);
    __syncthreads();
  } else {  // staged in Q, then widened into the Householder buffer
    tri_product<T, true>(Nm, L.ldn, r, dinv, Y, kCK, nullptr, Q, kQS);
    __syncthreads();
    for (int e = tid; e < r * kCK; e += kCT) {
      const int i = e >> 4, c = e & 15;
      if (c < k) Cq[i * 17 + c] = (U)Q[i * kQS + c];
    }
    __syncthreads();
  }
  // 3. Q = qr(C): FP64 CholeskyQR2 over the cluster (precision form), shifted
  //    CholeskyQR3 in FP32, or Householder in FP64 (their buffers live in Y, dead until
  //    step 4)
  if constexpr (P64) {
    double* S = reinterpret_cast<double*>(Y);
    double* pub = reinterpret_cast<double*>(buf);  // the pivot-row buffer is dead
    p64_cholqr_pass<T>(E, Q, r, k, i0, i1, false, S, S + 288, S + 304, Xg, pub);
    p64_cholqr_pass<T>(Q, Q, r, k, i0, i1, true, S, S + 288, S + 304, Xg, pub);
  } else if constexpr (sizeof(T) == 4) {
    cq3_f32(E, E, Q, r, k, reinterpret_cast<float*>(Y));
  } else {
    chol_householder<U, T>(Cq, 17, r, k, tau, Q);
  }
  // 4. E = N^T D^{-1} N Q
  tri_product<T, false>(Nm, L.ldn, r, nullptr, Q, kQS, dinv, Y, kCK);
  __syncthreads();
  tri_product<T, true>(Nm, L.ldn, r, nullptr, Y, kCK, nullptr, E, kQS);
  __syncthreads();
  // 5. D = E^T H over the own columns (k x w): a thread per (column, group of 4 rows of
  //    D) runs down the r rows of H, four sums in registers (a compact loop: this phase
  //    runs once per launch, so its code size, not its arithmetic, sets its time).  D may
  //    overwrite H's first k rows in place: it is written after a barrier, and the four
  //    threads of a column are always in the same round.
  if (h_smem) {
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
  }
  for (int rd = 0; rd < (4 * w + kCT - 1) / kCT; ++rd) {
    const int it = rd * kCT + tid, jj = it >> 2, cg = it & 3;
    const bool act = jj < w && 4 * cg < k;
    T acc[4] = {(T)0, (T)0, (T)0, (T)0};
    if (act) {
      const T* hp = Hsrc + jj;
      const T* ep = E + 4 * cg;
#pragma unroll 4
      for (int i = 0; i < r; ++i) {
        const T hv = hp[(long)i * ldh];
        T ev[4];
        V4<T>::ld(ep + i * kQS, ev);
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[e] = fma(ev[e], hv, acc[e]);
      }
    }
    __syncthreads();
    if (act) {
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (4 * cg + e < k) D[(long)(4 * cg + e) * ldd + jj] = acc[e];
    }
  }
  __syncthreads();
  // FP64 workspace of the precision form's eigen refinement and K's FP64 copy, in N (dead
  // after step 4)
  double* w64 = reinterpret_cast<double*>(Nm);
  double* Kd = w64 + kRefineWs;
  // K = D D^T: the own columns' part (4 threads per entry of the upper triangle), summed
  // over the cluster in rank order
  {
    T* Kp = reinterpret_cast<T*>(Xg);
    for (int e = tid; e < 4 * 136 + (kCT - (4 * 136) % kCT) % kCT; e += kCT) {
      const int pr = e >> 2, part = e & 3;
      T acc = 0;
      int ia = 0, ib = 0;
      if (pr < 136) {
        int rem = pr;
        while (rem >= kCK - ia) {
          rem -= kCK - ia;
          ++ia;
        }
        ib = ia + rem;
        if (ib < k)
          for (int t = part; t < w; t += 4) acc = fma(D[(long)ia * ldd + t], D[(long)ib * ldd + t], acc);
      }
      acc += __shfl_xor_sync(kAll, acc, 1);
      acc += __shfl_xor_sync(kAll, acc, 2);
      if (pr < 136 && part == 0) {
#pragma unroll
        for (int q = 0; q < kNC; ++q) cl_peer(Kp, q)[cr * 272 + ia * kCKs + ib] = acc;
      }
    }
    cl_sync();
    if (tid < kCK * kCK) {
      const int i = tid >> 4, j = tid & 15;
      const int lo = min(i, j), hi = max(i, j);
      T sum = 0;
      for (int q = 0; q < kNC; ++q) sum += Kp[q * 272 + lo * kCKs + hi];
      K0[i * kCKs + j] = sum;
      if constexpr (P64) Kd[i * 17 + j] = (double)sum;
    }
    __syncthreads();
  }
  // 6. eigen-decomposition of K: FP32 Jacobi on warps 0 .. 3, then the FP64 refinement in
  //    the precision form
  if (warp < kJW) {
    T* Kf = cj_jacobi<T>(K0, K1, V, 20);
    if (tid == 0) Kfin = Kf;
  }
  __syncthreads();
  T* Kf = Kfin;
  if constexpr (P64) p64_eig_refine<T>(Kd, V, Kf, w64);
  if (tid < kCK) order[tid] = tid;  // stays a valid index if a NaN breaks the ranking
  __syncthreads();
  // eigenvalues descending (rank by counting; ties keep index order); padded indices
  // (>= k) rank after the real ones
  if (tid < kCK) {
    const bool real = tid < k;
    const T l = Kf[tid * kCKs + tid];
    int rank = 0;
    for (int j = 0; j < kCK; ++j) {
      const T o = Kf[j * kCKs + j];
      const bool before = (j < k) ? (!real || o > l || (o == l && j < tid)) : (!real && j < tid);
      rank += before;
    }
    order[rank] = tid;
    if (real && !isfinite(l) && a.flag) atomicExch(a.flag, 1);
  }
  __syncthreads();
  // F = U_R / sigma (16 x 16 with zero rows >= k and columns >= R), CnT = Q U_R sigma
  for (int e = tid; e < kCK * kCK; e += kCT) {
    const int i = e >> 4, c = e & 15;
    T f = (T)0;
    if (c < R && i < k) {
      const T l = Kf[order[c] * kCKs + order[c]];
      const T sig = l > (T)0 ? sqrt(l) : (T)0;
      if (sig > (T)0) f = V[i * kCKs + order[c]] / sig;
    }
    F[i * kCK + c] = f;
  }
  if (cr == 0) {
    for (int e = tid; e < r * kCK; e += kCT) {
      const int i = e >> 4, c = e & 15;
      if (c >= R) continue;
      const T l = Kf[order[c] * kCKs + order[c]];
      const T sig = l > (T)0 ? sqrt(l) : (T)0;
      T acc = 0;
      for (int b = 0; b < k; ++b) acc = fma(Q[i * kQS + b], V[b * kCKs + order[c]], acc);
      CnTs[i * R + c] = acc * sig;
    }
  }
  __syncthreads();
  // 7. A = D^T F over the own columns (unsigned): a thread per (column, group of 4
  //    columns of A)
  for (int it = tid; it < 4 * w; it += kCT) {
    const int jj = it >> 2, cg = it & 3;
    if (4 * cg >= R) continue;
    T acc[4] = {(T)0, (T)0, (T)0, (T)0};
    for (int b = 0; b < k; ++b) {
      const T dv = D[(long)b * ldd + jj];
      T fv[4];
      V4<T>::ld(F + b * kCK + 4 * cg, fv);
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[e] = fma(dv, fv[e], acc[e]);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (4 * cg + e < R) Am[(long)jj * R + 4 * cg + e] = acc[e];
  }
  __syncthreads();
  // 8. canonical signs (largest-|.| entry of each column of A positive, lowest index on
  //    ties): each CTA's candidate over its columns, then the cluster's in rank order
  for (int c = warp; c < R; c += kCW) {
    T best = (T)-1;
    int bidx = 0x7fffffff;
    for (int i = lane; i < w; i += 32) {
      const T v = fabs(Am[(long)i * R + c]);
      if (v > best || (v == best && i < bidx)) {
        best = v;
        bidx = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ob = __shfl_xor_sync(kAll, best, o);
      const int oi = __shfl_xor_sync(kAll, bidx, o);
      if (ob > best || (ob == best && oi < bidx)) {
        best = ob;
        bidx = oi;
      }
    }
    if (lane == 0) {
      const T val = bidx < w ? Am[(long)bidx * R + c] : (T)0;
      const int gidx = bidx < w ? j0 + bidx : 0x7fffffff;
#pragma unroll
      for (int q = 0; q < kNC; ++q) {
        cl_peer(Xbest, q)[cr * kCK + c] = best;
        cl_peer(Xval, q)[cr * kCK + c] = val;
        cl_peer(Xidx, q)[cr * kCK + c] = gidx;
      }
    }
  }
  cl_sync();
  if (tid < R) {
    T best = (T)-1, val = (T)0;
    int bidx = 0x7fffffff;
    for (int q = 0; q < kNC; ++q) {
      const T b = Xbest[q * kCK + tid];
      const int ix = Xidx[q * kCK + tid];
      if (b > best || (b == best && ix < bidx)) {
        best = b;
        bidx = ix;
        val = Xval[q * kCK + tid];
      }
    }
    sgn[tid] = val < (T)0 ? (T)-1 : (T)1;
  }
  __syncthreads();
  for (int e = tid; e < w * R; e += kCT) {
    const int c = e % R;
    a.A_out[(long)j0 * R + e] = sgn[c] * Am[e];
  }
  if (cr == 0) {
    for (int e = tid; e < r * R; e += kCT) {
      const int rho = e / R, c = e - rho * R;
      const T v = sgn[c] * CnTs[e];
      if (a.CnT) a.CnT[e] = v;
      if (a.core) {
        long idx = 0, stride = 1, x = rho;
        for (int kk = a.map.order - 1; kk >= 0; --kk) {
          int digit;
          if (kk == a.map.n) {
            digit = c;
          } else {
            digit = (int)(x % a.map.ranks[kk]);
            x /= a.map.ranks[kk];
          }
          idx += digit * stride;
          stride *= a.map.ranks[kk];
        }
        a.core[idx] = v;
      }
    }
  }
}

template <typename T, typename U, bool P64>
__global__ void __cluster_dims__(kNC, 1, 1) __launch_bounds__(kCT, 1) k_lrls_chol(FusedArgs<T> a, bool h_smem) {
  pdl_trigger();
  pdl_wait();
  lrls_chol_body<T, U, P64>(a, h_smem);
}

// ---------------------------------------------------------------- small eigensolver

// K (n x n, n <= 16, symmetrised) = U Lambda U^T by the four-warp Jacobi above and, with
// P64, one FP64 refinement over the cluster; eigenvalues descending (ties in index
// order), sigma = sqrt(lambda).  Outputs as the general eigensolver's: Fm = U_R
// Sigma_R^{-1} and Uout = U_R (n x R), CnT = Q U_R Sigma_R (r x R; Q null: U_R Sigma_R,
// r = n); each may be null; CTA 0 writes them.  A non-finite eigenvalue sets *flag.
template <typename T, bool P64>
__global__ void __cluster_dims__(kNC, 1, 1) __launch_bounds__(kCT, 1)
    k_eig16(int n, int R, const T* __restrict__ K, const T* __restrict__ Q, int r,
            T* __restrict__ CnT, T* __restrict__ Fm, T* __restrict__ Uout, int* flag) {
  pdl_trigger();
  pdl_wait();
  __shared__ __align__(16) T K0[kCK * kCKs], K1[kCK * kCKs], V[kCK * kCKs];
  __shared__ __align__(16) double ws[P64 ? kRefineWs + kCK * 17 : 1];
  __shared__ int order[kCK];
  __shared__ T* Kfin;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid < kCK * kCK) {
    const int i = tid >> 4, j = tid & 15;
    const T v = (i < n && j < n) ? (T)0.5 * (K[i * n + j] + K[j * n + i]) : (T)0;
    K0[i * kCKs + j] = v;
    if constexpr (P64) ws[kRefineWs + i * 17 + j] = (double)v;
  }
  __syncthreads();
  if (warp < kJW) {
    T* Kf = cj_jacobi<T>(K0, K1, V, 20);
    if (tid == 0) Kfin = Kf;
  }
  __syncthreads();
  T* Kf = Kfin;
  if constexpr (P64) p64_eig_refine<T>(ws + kRefineWs, V, Kf, ws);
  if (tid < kCK) order[tid] = tid;  // stays a valid index if a NaN breaks the ranking
  __syncthreads();
  if (tid < kCK) {
    const bool real = tid < n;
    const T l = Kf[tid * kCKs + tid];
    int rank = 0;
    for (int j = 0; j < kCK; ++j) {
      const T o = Kf[j * kCKs + j];
      rank += (j < n) ? (!real || o > l || (o == l && j < tid)) : (!real && j < tid);
    }
    order[rank] = tid;
    if (real && !isfinite(l) && flag) atomicExch(flag, 1);
  }
  __syncthreads();
  if (cg::this_cluster().block_rank() != 0) return;
  for (int e = tid; e < n * R; e += kCT) {
    const int i = e / R, c = e - (e / R) * R;
    const T l = Kf[order[c] * kCKs + order[c]];
    const T sig = l > (T)0 ? sqrt(l) : (T)0;
    const T u = V[i * kCKs + order[c]];
    if (Fm) Fm[e] = sig > (T)0 ? u / sig : (T)0;
    if (Uout) Uout[e] = u;
  }
  if (CnT)
    for (int e = tid; e < r * R; e += kCT) {
      const int i = e / R, c = e - (e / R) * R;
      const T l = Kf[order[c] * kCKs + order[c]];
      const T sig = l > (T)0 ? sqrt(l) : (T)0;
      T acc;
      if (Q) {
        acc = 0;
        for (int a = 0; a < n; ++a) acc = fma(Q[(long)i * n + a], V[a * kCKs + order[c]], acc);
      } else {
        acc = V[i * kCKs + order[c]];
      }
      CnT[e] = acc * sig;
    }
}

template <typename T>
ts_status launch_eig16(int n, int R, const T* K, const T* Q, int r, T* CnT, T* Fm, T* Uout,
                       bool fp64, int* flag, cudaStream_t st) {
  if (n < 1 || n > kCK || R < 1 || R > n)
    return fail(TS_ERR_SHAPE, "eigensolver: n=%d R=%d outside 1 <= R <= n <= %d", n, R, kCK);
  if constexpr (sizeof(T) == 4) {
    if (fp64)
      return launch_pdl(k_eig16<T, true>, dim3(kNC), dim3(kCT), 0, st, n, R, K, Q, r, CnT, Fm,
                        Uout, flag);
  }
  return launch_pdl(k_eig16<T, false>, dim3(kNC), dim3(kCT), 0, st, n, R, K, Q, r, CnT, Fm, Uout,
                    flag);
}

template ts_status launch_eig16<float>(int, int, const float*, const float*, int, float*, float*,
                                       float*, bool, int*, cudaStream_t);
template ts_status launch_eig16<double>(int, int, const double*, const double*, int, double*,
                                        double*, double*, bool, int*, cudaStream_t);

// ---------------------------------------------------------------- host side

constexpr size_t kCholReserve = 1024;  // static shared memory of the kernel (~0.2 KB), with slack
// At least this much dynamic shared memory per CTA, so that no two CTAs of the cluster
// share an SM (their FP64 units and issue slots would be shared).
constexpr size_t kCholSpread = 120 * 1024;

// Layout of a subproblem: the own columns of H copied in when they fit (and A fits in
// H's rows below D), else D and A in shared memory when they fit, else in global memory.
static CholLayout chol_pick(int r, int s, int k, int R, size_t tsz, size_t usz) {
  const size_t cap = kMaxSmem - kCholReserve;
  if (R <= r - k) {
    CholLayout L = chol_layout(r, s, k, R, tsz, usz, true, false, false);
    if (L.total <= cap) return L;
  }
  CholLayout L = chol_layout(r, s, k, R, tsz, usz, false, true, true);
  if (L.total <= cap) return L;
  return chol_layout(r, s, k, R, tsz, usz, false, false, false);
}

bool lrls_chol_supported(int r, int s, int k, int R, int solve, size_t tsize, bool fp64) {
  if (solve != TS_SOLVE_RSVD || (fp64 && tsize == 8)) return false;
  if (r < 1 || s < 1 || R < 1 || k < R || k > kCK || r + k > kCMax) return false;
  if (tsize == 8 ? r > ElimShape<double>::NWE * ElimShape<double>::RS
                 : r > ElimShape<float>::NWE * ElimShape<float>::RS)
    return false;
  return chol_pick(r, s, k, R, tsize, tsize).total <= kMaxSmem - kCholReserve;
}

template <typename T>
ts_status launch_lrls_chol(const FusedArgs<T>& in, bool fp64, cudaStream_t st) {
  FusedArgs<T> a = in;
  const CholLayout L = chol_pick(a.r, a.s, a.k, a.R, sizeof(T), sizeof(T));
  a.m_smem = L.d_smem;
  const bool h = L.h_smem;
  const size_t bytes = L.total > kCholSpread ? L.total : kCholSpread;
  if constexpr (sizeof(T) == 4) {
    if (fp64) {  // the precision form: FP64 QR of C and FP64 refinement of K's eigenpairs
      TS_TRY(ensure_dynamic_smem((const void*)k_lrls_chol<T, T, true>, bytes));
      return launch_pdl(k_lrls_chol<T, T, true>, dim3(kNC), dim3(kCT), bytes, st, a, h);
    }
  }
  TS_TRY(ensure_dynamic_smem((const void*)k_lrls_chol<T, T, false>, bytes));
  return launch_pdl(k_lrls_chol<T, T, false>, dim3(kNC), dim3(kCT), bytes, st, a, h);
}

template ts_status launch_lrls_chol<float>(const FusedArgs<float>&, bool, cudaStream_t);
template ts_status launch_lrls_chol<double>(const FusedArgs<double>&, bool, cudaStream_t);

}  // namespace ts
