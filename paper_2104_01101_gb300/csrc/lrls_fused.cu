// The sketched rank-constrained least-squares subproblem (Sec. 4) in ONE thread block,
// after one multi-SM product has formed the augmented right-hand block
//   RSVD (Alg. 5):    [G | W | H] = Z^T [Z | Y Omega | Y]   (r x (r + k + s))
//   exact (Thm. 4.1): [G | H]     = Z^T [Z | Y]             (r x (r + s))
// Steps, all on chip:
//   1. Gauss-Jordan elimination of [G | W] (exact: [G | H]) with 16-wide panels: the
//      first r columns become G^{-1}, the rest C = G^{-1} W (exact: X = G^{-1} H).  G is
//      SPD (Z has full column rank), so no pivoting is needed.  Per panel one warp
//      inverts the 16 x 16 pivot block in registers -- the NEXT panel's, overlapped with
//      the current update -- while the other warps apply the rank-16 update in 8 x 2
//      register tiles: two block barriers per panel.
//   2. RSVD: Q = qr(C) by Householder reflections with warp c owning column c (one
//      barrier per reflector, then each warp forms its own column of Q); E = G^{-1} Q;
//      D = E^T H (= Q^T G^{-1} Z^T Y, k x s); K = D D^T.   Exact: M = X, K = X X^T.
//   3. K = U Lambda U^T by cyclic Jacobi with the whole block (round-robin pairs; each
//      round's rotations applied as one two-sided 2 x 2 block update while the next
//      round's rotations are formed; relative stopping rule with a rounding floor),
//      optionally polished by FP64 sweeps on V^T K V.
//   4. CnT = Q U_R Sigma_R (Q = I for exact), A = M^T U_R Sigma_R^{-1}, canonical column
//      signs (largest-magnitude entry of each column of A positive, lowest index on ties)
//      and C_(n)^T scattered into the core.
#include "dense_la.cuh"

namespace ts {

namespace {
constexpr int kThreads = 1024;
constexpr int kPb = 16;  // Gauss-Jordan panel width
constexpr int kPs = 20;  // row stride of the 16-wide panel buffers (16-byte aligned rows)
constexpr unsigned kFull = 0xffffffffu;
}  // namespace

__host__ __device__ inline int odd_ld(int n) { return n | 1; }
__host__ __device__ inline int quad_ld(int n) { return (n + 3) & ~3; }

// Shared-memory layout (byte offsets).  T = data type, U = QR type.
struct FusedLayout {
  int naug, lda, kq, ke, n;
  size_t A, P0, P1, rowold, colbuf, QA, Qo, Qt, tau, E, M, Kk, Vk, Am, Fm, CnTs, K64, V64, KV64,
      sched, memb, Kk2, K64b, total;
};

__host__ __device__ inline FusedLayout fused_layout(int r, int s, int k, int R, int solve,
                                                    size_t tsz, size_t usz, bool m_smem,
                                                    bool polish) {
  FusedLayout L{};
  const bool rsvd = solve == TS_SOLVE_RSVD;
  L.naug = r + (rsvd ? k : s);
  L.lda = odd_ld(L.naug);
  L.kq = odd_ld(k);
  L.ke = quad_ld(k);
  L.n = rsvd ? k : r;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    off = (off + 15) & ~(size_t)15;
    const size_t o = off;
    off += bytes;
    return o;
  };
  const size_t r8 = (size_t)((r + 7) & ~7);
  L.A = take(tsz * (size_t)r * L.lda);
  L.P0 = take(tsz * kPb * kPs);
  L.P1 = take(tsz * kPb * kPs);
  L.rowold = take(tsz * kPb * (size_t)L.lda);
  L.colbuf = take(tsz * (r8 + 8) * kPs);  // + 8 rows: the last 10-row update item's overhang
  L.QA = take(rsvd ? usz * (size_t)r * L.kq : 0);
  L.Qo = take(rsvd ? usz * (size_t)r * L.kq : 0);
  L.Qt = take(rsvd ? tsz * (size_t)r * L.ke : 0);
  L.tau = take(rsvd ? usz * (size_t)k : 0);
  L.E = take(rsvd ? tsz * (size_t)r * L.ke : 0);
  L.M = take(rsvd && m_smem ? tsz * (size_t)k * s : 0);
  L.Kk = take(tsz * (size_t)L.n * L.n);
  L.Vk = take(tsz * (size_t)L.n * L.n);
  L.Am = take(m_smem ? tsz * (size_t)s * R : 0);
  L.Fm = take(tsz * (size_t)L.n * R);
  L.CnTs = take(tsz * (size_t)r * R);
  L.K64 = take(polish ? 8 * (size_t)L.n * L.n : 0);
  L.V64 = take(polish ? 8 * (size_t)L.n * L.n : 0);
  L.KV64 = take(polish ? 8 * (size_t)L.n * L.n : 0);
  const int np = (L.n + 1) & ~1;
  L.sched = take(sizeof(int) * (size_t)(np - 1) * (np / 2));
  L.memb = take(sizeof(int) * (size_t)(np - 1) * np);
  L.Kk2 = take(tsz * (size_t)L.n * L.n);
  L.K64b = take(polish ? 8 * (size_t)L.n * L.n : 0);
  L.total = off;
  return L;
}

__device__ __forceinline__ void load4(const float* p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x;
  v[1] = t.y;
  v[2] = t.z;
  v[3] = t.w;
}
__device__ __forceinline__ void load4(const double* p, double (&v)[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p);
  const double2 b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}

// ---------------------------------------------------------------- Gauss-Jordan

// Inverse of a 16 x 16 SPD block held in registers by one warp: lane l owns row (l & 15),
// columns 8 (l >> 4) .. 8 (l >> 4) + 7.  Gauss-Jordan without pivoting, pivot row and
// column exchanged by shuffles; a non-positive or non-finite pivot sets *flag and is
// replaced by 1.
template <typename T>
__device__ __forceinline__ void warp_inverse16(T (&a)[8], int* flag) {
  const int lane = threadIdx.x & 31, i = lane & 15, h = lane >> 4;
#pragma unroll
  for (int q = 0; q < kPb; ++q) {
    T piv = __shfl_sync(kFull, a[q & 7], q + 16 * (q >> 3));
    if (!(piv > (T)0) || !isfinite(piv)) {
      if (lane == 0 && flag) atomicExch(flag, 1);
      piv = (T)1;
    }
    const T inv = (T)1 / piv;
    const T f = __shfl_sync(kFull, a[q & 7], i + 16 * (q >> 3)) * inv;
    T aq[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) aq[t] = __shfl_sync(kFull, a[t], q + 16 * h);
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const bool colq = (h == (q >> 3)) && (t == (q & 7));
      if (i == q) a[t] = colq ? inv : aq[t] * inv;
      else a[t] = colq ? -f : a[t] - f * aq[t];
    }
  }
}

// One RPI-row x 2-column tile per lane (columns jb and jb + 32) of the panel update,
// with L = colbuf holding -A21 P on rows outside the panel and P on the panel rows:
// rows of the panel: A <- P A_panel (A11 <- P); rows outside: A <- A + L rowold
// (A21 <- L).  The next panel's pivot block is left to warp 0.  Rows are classified one
// by one (an item may straddle the panel's 16-row boundary).
template <typename T, int RPI>
__device__ __forceinline__ void gj_update_tile(T* A, int r, int ncol, int lda, int i0, int jb,
                                               int p0, int nb, int q0, int nbn,
                                               const T* rowold, const T* L) {
  const int jc[2] = {jb, jb + 32};
  bool valid[2], pcol[2], ncolq[2];
#pragma unroll
  for (int x = 0; x < 2; ++x) {
    valid[x] = jc[x] < ncol;
    pcol[x] = jc[x] >= p0 && jc[x] < p0 + nb;
    ncolq[x] = nbn > 0 && jc[x] >= q0 && jc[x] < q0 + nbn;
  }
  T acc[2][RPI];
#pragma unroll
  for (int rr = 0; rr < RPI; ++rr) {
    const int i = i0 + rr;
    const bool keep = (i < p0 || i >= p0 + kPb) && i < r;
#pragma unroll
    for (int x = 0; x < 2; ++x) acc[x][rr] = (keep && valid[x]) ? A[i * lda + jc[x]] : (T)0;
  }
  const T* Lrow = L + i0 * kPs;
#pragma unroll 1
  for (int u = 0; u < kPb; u += 4) {
    T b[2][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int x = 0; x < 2; ++x) b[x][q] = valid[x] ? rowold[(u + q) * lda + jc[x]] : (T)0;
#pragma unroll
    for (int rr = 0; rr < RPI; ++rr) {
      T l4[4];
      load4(Lrow + rr * kPs + u, l4);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[0][rr] += l4[q] * b[0][q];
        acc[1][rr] += l4[q] * b[1][q];
      }
    }
  }
#pragma unroll
  for (int rr = 0; rr < RPI; ++rr) {
    const int i = i0 + rr;
    if (i >= r) break;
    const bool in_next = nbn > 0 && i >= q0 && i < q0 + kPb;
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      if (!valid[x] || (in_next && ncolq[x])) continue;
      A[i * lda + jc[x]] = pcol[x] ? Lrow[rr * kPs + (jc[x] - p0)] : acc[x][rr];
    }
  }
}

// In-place Gauss-Jordan elimination of the augmented block [G | B] (r x ncol, row stride
// lda, ncol >= r): on exit the first r columns hold G^{-1}, the others G^{-1} B.  Panel
// step with P = A11^{-1} ("1" = the 16 panel rows / columns):
//   A11 <- P,  A12 <- P A12,  A21 <- -A21 P,  A22 <- A22 - A21 P A12.
template <typename T>
__device__ void gauss_jordan(T* A, int r, int ncol, int lda, T* P0, T* P1, T* rowold, T* colbuf,
                             int* flag) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthr = blockDim.x, nwarp = nthr >> 5;
  const int li = lane & 15, lh = lane >> 4;
  if (warp == 0) {
    const int nb = min(kPb, r);
    T a8[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int j = lh * 8 + t;
      a8[t] = (li < nb && j < nb) ? A[li * lda + j] : (li == j ? (T)1 : (T)0);
    }
    warp_inverse16<T>(a8, flag);
#pragma unroll
    for (int t = 0; t < 8; ++t) P0[li * kPs + lh * 8 + t] = a8[t];
  }
  __syncthreads();
  // rows per update item: the fewest that give every update warp at most one item
  const int nw3 = nwarp - nwarp / 4;
  const int nc64 = (ncol + 63) / 64;
  const int r8 = (r + 7) & ~7;  // colbuf rows (the buffer's extent)
  const int rpi = ((r + 7) / 8) * nc64 <= nw3 ? 8 : ((r + 9) / 10) * nc64 <= nw3 ? 10 : 8;
  const int nitems = ((r + rpi - 1) / rpi) * nc64;
  int pb = 0;
  for (int p0 = 0; p0 < r; p0 += kPb, pb ^= 1) {
    const int nb = min(kPb, r - p0);
    const T* P = pb ? P1 : P0;
    T* Pn = pb ? P0 : P1;
    // (a) the panel rows as they are, and colbuf = -A21 P
    for (int e = tid; e < kPb * ncol; e += nthr) {
      const int t = e / ncol, j = e - t * ncol;
      rowold[t * lda + j] = t < nb ? A[(p0 + t) * lda + j] : (T)0;
    }
    for (int e = tid; e < r8 * kPb; e += nthr) {
      const int i = e >> 4, u = e & 15;
      if (i >= p0 && i < p0 + kPb) {  // the panel rows: P itself
        colbuf[i * kPs + u] = P[(i - p0) * kPs + u];
        continue;
      }
      T acc0 = 0, acc1 = 0;  // two chains; t >= nb reads stay inside the row (masked)
      if (u < nb && i < r) {
        const T* Ai = A + i * lda + p0;
#pragma unroll
        for (int t = 0; t < kPb; t += 2) {
          if (t < nb) acc0 += Ai[t] * P[t * kPs + u];
          if (t + 1 < nb) acc1 += Ai[t + 1] * P[(t + 1) * kPs + u];
        }
      }
      colbuf[i * kPs + u] = -(acc0 + acc1);
    }
    __syncthreads();
    // (b) rank-nb update; warp 0 forms and inverts the next pivot block
    const int q0 = p0 + kPb;
    const int nbn = q0 < r ? min(kPb, r - q0) : 0;
    if (warp == 0) {
      if (nbn > 0) {
        const int i = q0 + li;
        T ci[kPb];
#pragma unroll
        for (int u = 0; u < kPb; u += 4)
          load4(colbuf + i * kPs + u, *reinterpret_cast<T(*)[4]>(ci + u));
        T a8[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int jl = lh * 8 + t;
          T v = (li == jl) ? (T)1 : (T)0;
          if (li < nbn && jl < nbn) {
            const int j = q0 + jl;
            v = A[i * lda + j];
#pragma unroll
            for (int u = 0; u < kPb; ++u) v += ci[u] * rowold[u * lda + j];
          }
          a8[t] = v;
        }
        warp_inverse16<T>(a8, flag);
#pragma unroll
        for (int t = 0; t < 8; ++t) Pn[li * kPs + lh * 8 + t] = a8[t];
      }
    } else if ((warp & 3) != 0) {
      // The update runs on the warps of the other three SM sub-partitions (warp w on
      // sub-partition w % 4), so that warp 0's dependent chain is not starved of issue slots.
      const int w3 = (warp >> 2) * 3 + (warp & 3) - 1;
      for (int it = w3; it < nitems; it += nw3) {
        const int i0 = (it / nc64) * rpi, jb = (it % nc64) * 64 + lane;
        if (rpi == 8)
          gj_update_tile<T, 8>(A, r, ncol, lda, i0, jb, p0, nb, q0, nbn, rowold, colbuf);
        else
          gj_update_tile<T, 10>(A, r, ncol, lda, i0, jb, p0, nb, q0, nbn, rowold, colbuf);
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- Householder QR

// Thin QR of A (r x k, row stride lda, type U) by Householder reflections, warp c owning
// column c (k <= warps of the block).  On exit A holds the reflectors (v_j(j) in A(j, j))
// and Qo (r x k, row stride lda) the orthonormal factor.  A zero column gives tau = 0.
template <typename U>
__device__ void householder_warps(U* A, U* Qo, U* tau, int r, int k, int lda) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int j = 0; j < k; ++j) {
    if (warp == j) {
      __syncwarp();
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
      U w = 0;
      for (int i = j + lane; i < r; i += 32) w += A[i * lda + j] * A[i * lda + warp];
      w = warp_sum(w) * tj;
      for (int i = j + lane; i < r; i += 32) A[i * lda + warp] -= w * A[i * lda + j];
    }
  }
  __syncthreads();
  if (warp < k) {  // Q(:, c) = H_0 ... H_c e_c, since H_j e_c = e_c for j > c
    const int c = warp;
    for (int i = lane; i < r; i += 32) Qo[i * lda + c] = (i == c) ? (U)1 : (U)0;
    __syncwarp();
    for (int j = c; j >= 0; --j) {
      const U tj = tau[j];
      U w = 0;
      for (int i = j + lane; i < r; i += 32) w += A[i * lda + j] * Qo[i * lda + c];
      w = warp_sum(w) * tj;
      for (int i = j + lane; i < r; i += 32) Qo[i * lda + c] -= w * A[i * lda + j];
      __syncwarp();
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- Jacobi eigensolver

template <typename U>
__host__ __device__ constexpr U jacobi_tol() {
  return sizeof(U) == 4 ? (U)4.8e-7 : (U)8.9e-16;  // 8 unit roundoffs
}
template <typename U>
__host__ __device__ constexpr U jacobi_floor() {
  return sizeof(U) == 4 ? (U)1.2e-7 : (U)2.2e-16;  // 2 unit roundoffs
}

// Round-robin schedule of cyclic Jacobi for order n (n <= 64): np - 1 rounds of np / 2
// disjoint pairs (np = n rounded up to even), pair (p, q) packed as p | q << 8 with
// q = 255 for the padding index.
// memb[t * np + a] = 2 i + (a is the second index of its pair) for the pair i of round t
// that holds index a.
__device__ void jacobi_schedule(int n, int* sched, int* memb) {
  const int np = (n + 1) & ~1, npairs = np >> 1, nrounds = np - 1;
  for (int e = threadIdx.x; e < nrounds * npairs; e += blockDim.x) {
    const int t = e / npairs, i = e - t * npairs;
    const int a = i == 0 ? t : (t + i) % nrounds;
    const int b = i == 0 ? nrounds : (t - i + nrounds) % nrounds;
    const int p = min(a, b), q = max(a, b);
    sched[e] = p | ((q < n ? q : 255) << 8);
    memb[t * np + p] = 2 * i;
    memb[t * np + q] = 2 * i + 1;
  }
}

__device__ __forceinline__ float fast_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fast_div(double a, double b) { return a / b; }
// 1 / sqrt(x) to working precision (one Newton step on the FP32 approximation)
__device__ __forceinline__ float unit_rsqrt(float x) {
  const float r = rsqrtf(x);
  return r * (1.5f - 0.5f * x * r * r);
}
__device__ __forceinline__ double unit_rsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float fast_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double fast_rsqrt(double x) { return rsqrt(x); }

// Rotation of pair pq (packed as in jacobi_schedule) for the current matrix A: J =
// [[c, s], [-s, c]] on (p, q) makes (J^T A J)(p, q) zero; identity (rot = false) when
// |a_pq| is below the relative and the absolute thresholds, or for the padding index.
template <typename U>
__device__ __forceinline__ void jacobi_rotation(const U* A, int n, int pq, U tol2, U floor_abs,
                                                int& p, int& q, U& c, U& s, bool& rot) {
  p = pq & 255;
  q = (pq >> 8) == 255 ? -1 : (pq >> 8);
  c = 1;
  s = 0;
  rot = false;
  if (q < 0) return;
  const U apq = A[p * n + q], app = A[p * n + p], aqq = A[q * n + q];
  if (apq * apq > tol2 * fabs(app * aqq) && fabs(apq) > floor_abs) {
    // t = sign(theta) / (|theta| + sqrt(theta^2 + 1)); its rounding only perturbs the angle,
    // while c = (1 + t^2)^(-1/2) to working precision keeps the rotation orthogonal
    const U theta = fast_div(aqq - app, 2 * apq);
    const U h = theta * theta + 1;
    const U tt = fast_div(theta >= (U)0 ? (U)1 : (U)-1, fabs(theta) + h * fast_rsqrt(h));
    c = unit_rsqrt(tt * tt + 1);
    s = tt * c;
    rot = true;
  }
}

// The 2 x 2 block of J^T A J on rows {p1, q1} x columns {p2, q2} for the rotations
// J = [[c, s], [-s, c]] of the two pairs (q < 0: padding index, entries zero).  The
// products are written as explicit fused multiply-adds so that every caller obtains the
// same rounded values.
template <typename U>
__device__ __forceinline__ void rotate_block(const U* A, int n, int p1, int q1, U c1, U s1,
                                             int p2, int q2, U c2, U s2, U& n00, U& n01,
                                             U& n10, U& n11) {
  const U b00 = A[p1 * n + p2];
  const U b01 = q2 >= 0 ? A[p1 * n + q2] : (U)0;
  const U b10 = q1 >= 0 ? A[q1 * n + p2] : (U)0;
  const U b11 = (q1 >= 0 && q2 >= 0) ? A[q1 * n + q2] : (U)0;
  const U t00 = fma(c1, b00, -(s1 * b10)), t01 = fma(c1, b01, -(s1 * b11));
  const U t10 = fma(s1, b00, c1 * b10), t11 = fma(s1, b01, c1 * b11);
  n00 = fma(c2, t00, -(s2 * t01));
  n01 = fma(s2, t00, c2 * t01);
  n10 = fma(c2, t10, -(s2 * t11));
  n11 = fma(s2, t10, c2 * t11);
}

// Rotation parameters of one round (np / 2 <= 32 pairs), double-buffered.
template <typename U>
struct JacobiRound {
  int p[2][kMaxEig / 2 + 1], q[2][kMaxEig / 2 + 1];
  U c[2][kMaxEig / 2 + 1], s[2][kMaxEig / 2 + 1];
};

// Cyclic Jacobi by the whole block on the symmetric n x n matrix in A (row stride n,
// n <= 64), double-buffered with A2; V (n x n) accumulates the rotations onto its start
// basis.  Each round applies its rotations (J = [[c, s], [-s, c]] on each pair of the
// round-robin schedule) as one update of the 2 x 2 blocks of J^T A J into the other
// buffer, plus V J.  The rotations of the NEXT round are computed at the same time by
// threads without items: the three entries they need are formed from the current buffer
// and this round's rotations with the same arithmetic as the block update, so one
// barrier per round suffices.  A pair rotates when |a_pq| exceeds both tol sqrt(|a_pp
// a_qq|) (relative accuracy) and floor_rel max_i |a_ii| (the rounding level of A); the
// loop ends after a sweep without rotations or after max_sweeps (<= 31).  sched and memb
// come from jacobi_schedule.  Returns the buffer holding the result.
template <typename U>
__device__ U* block_jacobi(U* A, U* A2, U* V, int n, U tol, U floor_rel, int max_sweeps,
                           const int* sched, const int* memb, JacobiRound<U>& rd, int* flags,
                           int* smax, U* red) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int np = (n + 1) & ~1, npairs = np >> 1, nrounds = np - 1;
  if (tid < 32) {
    U d = 0;
    for (int i = tid; i < n; i += 32) d = fmax(d, fabs(A[i * n + i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) d = fmax(d, __shfl_xor_sync(kFull, d, o));
    if (tid == 0) red[0] = d;
  }
  for (int i = tid; i < 32; i += nthr) {
    flags[i] = 0;
    smax[i] = 0;
  }
  __syncthreads();
  const U floor_abs = floor_rel * red[0], tol2 = tol * tol;
  // A sweep whose largest rotation has |s| <= sqrt(tol) ends the loop: Jacobi converges
  // quadratically, so the next sweep's angles would be ~tol, below the rotation test.
  const float stop_s = (float)sqrt(tol);
  const int nblk = npairs * npairs, nitems = nblk + n * npairs;
  // rotation threads: the last npairs threads (they own no item when the block is large)
  const int rbase = nthr - npairs;
  const bool rthread = tid >= rbase;
  const int ri = tid - rbase;
  if (tid < npairs) {  // rotations of round 0 from the start matrix
    int p, q;
    U c, s;
    bool rot;
    jacobi_rotation<U>(A, n, sched[tid], tol2, floor_abs, p, q, c, s, rot);
    rd.p[0][tid] = p;
    rd.q[0][tid] = q;
    rd.c[0][tid] = c;
    rd.s[0][tid] = s;
    if (rot) {
      flags[0] = 1;
      atomicMax(&smax[0], __float_as_int((float)fabs(s)));
    }
  }
  __syncthreads();
  U* Ao = A;
  U* An = A2;
  int cur = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int t = 0; t < nrounds; ++t) {
      const int* rp = rd.p[cur];
      const int* rq = rd.q[cur];
      const U* rc = rd.c[cur];
      const U* rs = rd.s[cur];
      for (int e = tid; tid < rbase && e < nitems; e += rbase) {
        if (e < nblk) {
          const int i = e / npairs, j = e - (e / npairs) * npairs;
          const int p1 = rp[i], q1 = rq[i], p2 = rp[j], q2 = rq[j];
          U n00, n01, n10, n11;
          rotate_block<U>(Ao, n, p1, q1, rc[i], rs[i], p2, q2, rc[j], rs[j], n00, n01, n10, n11);
          An[p1 * n + p2] = n00;
          if (q2 >= 0) An[p1 * n + q2] = n01;
          if (q1 >= 0) An[q1 * n + p2] = n10;
          if (q1 >= 0 && q2 >= 0) An[q1 * n + q2] = n11;
        } else {
          const int f = e - nblk;
          const int l = f / npairs, j = f - (f / npairs) * npairs;
          const int p2 = rp[j], q2 = rq[j];
          const U c2 = rc[j], s2 = rs[j];
          if (q2 >= 0 && s2 != (U)0) {
            const U vp = V[l * n + p2], vq = V[l * n + q2];
            V[l * n + p2] = c2 * vp - s2 * vq;
            V[l * n + q2] = s2 * vp + c2 * vq;
          }
        }
      }
      if (rthread) {  // rotation of pair ri for the next round, from J^T Ao J
        const int tn = t + 1 < nrounds ? t + 1 : 0;
        const int sn = t + 1 < nrounds ? sweep : sweep + 1;
        const int pq = sched[tn * npairs + ri];
        const int p = pq & 255, q = (pq >> 8) == 255 ? -1 : (pq >> 8);
        U c = 1, s = 0;
        if (q >= 0) {
          const int ma = memb[t * np + p], mb = memb[t * np + q];
          const int ia = ma >> 1, ib = mb >> 1, ra = ma & 1, rb = mb & 1;
          U x00, x01, x10, x11, y00, y01, y10, y11, z00, z01, z10, z11;
          rotate_block<U>(Ao, n, rp[ia], rq[ia], rc[ia], rs[ia], rp[ia], rq[ia], rc[ia], rs[ia],
                          x00, x01, x10, x11);
          rotate_block<U>(Ao, n, rp[ib], rq[ib], rc[ib], rs[ib], rp[ib], rq[ib], rc[ib], rs[ib],
                          y00, y01, y10, y11);
          rotate_block<U>(Ao, n, rp[ia], rq[ia], rc[ia], rs[ia], rp[ib], rq[ib], rc[ib], rs[ib],
                          z00, z01, z10, z11);
          const U app = ra ? x11 : x00, aqq = rb ? y11 : y00;
          const U apq = ra ? (rb ? z11 : z10) : (rb ? z01 : z00);
          if (apq * apq > tol2 * fabs(app * aqq) && fabs(apq) > floor_abs) {
            const U theta = fast_div(aqq - app, 2 * apq);
            const U h = theta * theta + 1;
            const U tt =
                fast_div(theta >= (U)0 ? (U)1 : (U)-1, fabs(theta) + h * fast_rsqrt(h));
            c = unit_rsqrt(tt * tt + 1);
            s = tt * c;
            if (sn < 32) {
              flags[sn] = 1;
              atomicMax(&smax[sn], __float_as_int((float)fabs(s)));
            }
          }
        }
        rd.p[cur ^ 1][ri] = p;
        rd.q[cur ^ 1][ri] = q;
        rd.c[cur ^ 1][ri] = c;
        rd.s[cur ^ 1][ri] = s;
      }
      U* tmp = Ao;
      Ao = An;
      An = tmp;
      cur ^= 1;
      __syncthreads();
    }
    if (!flags[sweep] || __int_as_float(smax[sweep]) <= stop_s) break;
  }
  return Ao;
}

// ---------------------------------------------------------------- the kernel

template <typename T, typename U, bool POLISH64>
__device__ __forceinline__ void lrls_fused_body(const FusedArgs<T>& a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ JacobiRound<T> jround;
  __shared__ JacobiRound<double> jround64;
  __shared__ int jflags[32], jsmax[32];
  __shared__ T jred[1];
  __shared__ double jred64[1];
  __shared__ int order[kMaxEig];
  __shared__ T sgn[kMaxEig];
  const int r = a.r, s = a.s, k = a.k, R = a.R;
  const bool rsvd = a.solve == TS_SOLVE_RSVD;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nthr = blockDim.x, nwarp = nthr >> 5;
  const FusedLayout L = fused_layout(r, s, k, R, a.solve, sizeof(T), sizeof(U), a.m_smem, POLISH64);
  const int lda = L.lda, naug = L.naug, n = L.n, kq = L.kq, ke = L.ke;
  T* A = reinterpret_cast<T*>(smem_raw + L.A);
  T* P0 = reinterpret_cast<T*>(smem_raw + L.P0);
  T* P1 = reinterpret_cast<T*>(smem_raw + L.P1);
  T* rowold = reinterpret_cast<T*>(smem_raw + L.rowold);
  T* colbuf = reinterpret_cast<T*>(smem_raw + L.colbuf);
  U* QA = reinterpret_cast<U*>(smem_raw + L.QA);
  U* Qo = reinterpret_cast<U*>(smem_raw + L.Qo);
  T* Qt = reinterpret_cast<T*>(smem_raw + L.Qt);
  U* tau = reinterpret_cast<U*>(smem_raw + L.tau);
  T* E = reinterpret_cast<T*>(smem_raw + L.E);
  T* Kk = reinterpret_cast<T*>(smem_raw + L.Kk);
  T* Vk = reinterpret_cast<T*>(smem_raw + L.Vk);
  T* Am = a.m_smem ? reinterpret_cast<T*>(smem_raw + L.Am) : a.A_out;
  T* Fm = reinterpret_cast<T*>(smem_raw + L.Fm);
  T* CnTs = reinterpret_cast<T*>(smem_raw + L.CnTs);

  // 1. stage the augmented block and run Gauss-Jordan
  for (int e = tid; e < r * naug; e += nthr) {
    const int i = e / naug, j = e - i * naug;
    T v;
    if (j < r) v = a.G[i * a.ldg + j];
    else if (rsvd) v = a.W[i * a.ldw + (j - r)];
    else v = a.H[i * a.ldh + (j - r)];
    A[i * lda + j] = v;
  }
  __syncthreads();
  gauss_jordan<T>(A, r, naug, lda, P0, P1, rowold, colbuf, a.flag);

  const T* M;  // n x s, row stride ldm: the matrix whose Gram K is decomposed
  int ldm;
  if (rsvd) {
    // 2. Q = qr(C), C = A(:, r:r+k)
    for (int e = tid; e < r * k; e += nthr) {
      const int i = e / k, c = e - i * k;
      QA[i * kq + c] = (U)A[i * lda + r + c];
    }
    __syncthreads();
    householder_warps<U>(QA, Qo, tau, r, k, kq);
    for (int e = tid; e < r * ke; e += nthr) {
      const int i = e / ke, c = e - i * ke;
      Qt[e] = c < k ? (T)Qo[i * kq + c] : (T)0;
    }
    __syncthreads();
    // 3. E = G^{-1} Q (thread per row and group of 8 columns)
    const int ng = (ke + 7) >> 3;
    for (int e = tid; e < r * ng; e += nthr) {
      const int i = e / ng, c0 = 8 * (e - (e / ng) * ng);
      const bool two = c0 + 4 < ke;
      T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll 4
      for (int l = 0; l < r; ++l) {
        const T g = A[i * lda + l];
        T v[4], w[4];
        load4(Qt + l * ke + c0, v);
        if (two) load4(Qt + l * ke + c0 + 4, w);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          acc[c] += g * v[c];
          if (two) acc[4 + c] += g * w[c];
        }
      }
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (c < 4 || two) E[i * ke + c0 + c] = acc[c];
    }
    // 4. D = E^T H (k x s): a thread streams one column of H over half of the rows; the
    //    two halves are added onto zero, an order-independent sum.
    T* D = a.m_smem ? reinterpret_cast<T*>(smem_raw + L.M) : a.Mbuf;
    const int halves = (2 * s <= nthr) ? 2 : 1;
    if (halves == 2)
      for (int e = tid; e < k * s; e += nthr) D[e] = (T)0;
    __syncthreads();
    const int rh = (r + halves - 1) / halves;
    for (int e = tid; e < s * halves; e += nthr) {
      const int part = e / s, j = e - part * s;
      const int i0 = part * rh, i1 = min(r, i0 + rh);
      for (int c0 = 0; c0 < k; c0 += 16) {
        T acc[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = 0;
        for (int i = i0; i < i1; i += 8) {  // 8 loads of H in flight per thread
          T hv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) hv[u] = (i + u < i1) ? a.H[(long)(i + u) * a.ldh + j] : (T)0;
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int ii = min(i + u, i1 - 1);  // past i1 the weight hv[u] is zero
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              if (c0 + 4 * q < ke) {
                T v[4];
                load4(E + ii * ke + c0 + 4 * q, v);
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[4 * q + c] += v[c] * hv[u];
              }
            }
          }
        }
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          if (c0 + c >= k) break;
          T* dst = D + (long)(c0 + c) * s + j;
          if (halves == 2) atomicAdd(dst, acc[c]);
          else *dst = acc[c];
        }
      }
    }
    M = D;
    ldm = s;
  } else {
    M = A + r;  // X = G^{-1} H
    ldm = lda;
  }
  __syncthreads();
  // 5. K = M M^T (upper triangle by warps, mirrored), V = I
  for (int pr = warp; pr < n * n; pr += nwarp) {
    const int i = pr / n, j = pr - (pr / n) * n;
    if (j < i) continue;
    T acc = 0;
    for (int t = lane; t < s; t += 32) acc += M[(long)i * ldm + t] * M[(long)j * ldm + t];
    acc = warp_sum(acc);
    if (lane == 0) {
      Kk[i * n + j] = acc;
      Kk[j * n + i] = acc;
    }
  }
  for (int e = tid; e < n * n; e += nthr) Vk[e] = (e / n == e % n) ? (T)1 : (T)0;
  __syncthreads();
  // 6. eigen-decomposition of K (optionally polished in FP64 on V^T K V, K formed in FP64)
  int* sched = reinterpret_cast<int*>(smem_raw + L.sched);
  int* memb = reinterpret_cast<int*>(smem_raw + L.memb);
  jacobi_schedule(n, sched, memb);
  __syncthreads();
  T* Kf = block_jacobi<T>(Kk, reinterpret_cast<T*>(smem_raw + L.Kk2), Vk, n, jacobi_tol<T>(),
                          jacobi_floor<T>(), 20, sched, memb, jround, jflags, jsmax, jred);
  if constexpr (POLISH64) {
    double* K64 = reinterpret_cast<double*>(smem_raw + L.K64);
    double* V64 = reinterpret_cast<double*>(smem_raw + L.V64);
    double* KV = reinterpret_cast<double*>(smem_raw + L.KV64);
    for (int pr = warp; pr < n * n; pr += nwarp) {
      const int i = pr / n, j = pr - (pr / n) * n;
      if (j < i) continue;
      double acc = 0;
      for (int t = lane; t < s; t += 32)
        acc += (double)M[(long)i * ldm + t] * (double)M[(long)j * ldm + t];
      acc = warp_sum(acc);
      if (lane == 0) {
        K64[i * n + j] = acc;
        K64[j * n + i] = acc;
      }
    }
    for (int e = tid; e < n * n; e += nthr) V64[e] = (double)Vk[e];
    __syncthreads();
    for (int e = tid; e < n * n; e += nthr) {
      const int i = e / n, j = e - (e / n) * n;
      double acc = 0;
      for (int b = 0; b < n; ++b) acc += K64[i * n + b] * V64[b * n + j];
      KV[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += nthr) {
      const int i = e / n, j = e - (e / n) * n;
      double acc = 0;
      for (int b = 0; b < n; ++b) acc += V64[b * n + i] * KV[b * n + j];
      K64[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += nthr) {
      const int i = e / n, j = e - (e / n) * n;
      if (i < j) {
        const double v = 0.5 * (K64[i * n + j] + K64[j * n + i]);
        K64[i * n + j] = v;
        K64[j * n + i] = v;
      }
    }
    __syncthreads();
    const double* Kf64 = block_jacobi<double>(
        K64, reinterpret_cast<double*>(smem_raw + L.K64b), V64, n, jacobi_tol<double>(),
        jacobi_floor<double>(), 10, sched, memb, jround64, jflags, jsmax, jred64);
    for (int e = tid; e < n * n; e += nthr) Vk[e] = (T)V64[e];
    if (tid < n) Kf[tid * n + tid] = (T)Kf64[tid * n + tid];
    __syncthreads();
  }
  // 7. eigenvalues descending (rank by counting; ties keep index order)
  if (tid < n) order[tid] = tid;
  __syncthreads();
  if (tid < n) {
    const T l = Kf[tid * n + tid];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const T o = Kf[j * n + j];
      rank += (o > l) || (o == l && j < tid);
    }
    if (rank < n) order[rank] = tid;
    if (!isfinite(l) && a.flag) atomicExch(a.flag, 1);
  }
  __syncthreads();
  // 8. Fm = U_R / sigma;  CnT = Q U_R sigma (Q = I for exact)
  for (int e = tid; e < n * R; e += nthr) {
    const int i = e / R, c = e - (e / R) * R;
    const T l = Kf[order[c] * n + order[c]];
    const T sig = l > (T)0 ? sqrt(l) : (T)0;
    Fm[e] = sig > (T)0 ? Vk[i * n + order[c]] / sig : (T)0;
  }
  for (int e = tid; e < r * R; e += nthr) {
    const int i = e / R, c = e - (e / R) * R;
    const T l = Kf[order[c] * n + order[c]];
    const T sig = l > (T)0 ? sqrt(l) : (T)0;
    T acc;
    if (rsvd) {
      acc = 0;
      for (int b = 0; b < k; ++b) acc += Qt[i * ke + b] * Vk[b * n + order[c]];
    } else {
      acc = Vk[i * n + order[c]];
    }
    CnTs[e] = acc * sig;
  }
  __syncthreads();
  // 9. A = M^T Fm (unsigned), 8 columns per thread
  const int ng = (R + 7) / 8;
  for (int e = tid; e < s * ng; e += nthr) {
    const int g = e / s, j = e - g * s;
    T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = 0; b < n; ++b) {
      const T mv = M[(long)b * ldm + j];
#pragma unroll
      for (int c = 0; c < 8; ++c)
        if (8 * g + c < R) acc[c] += mv * Fm[b * R + 8 * g + c];
    }
#pragma unroll
    for (int c = 0; c < 8; ++c)
      if (8 * g + c < R) Am[(long)j * R + 8 * g + c] = acc[c];
  }
  __syncthreads();
  // 10. canonical signs, then the signed outputs and the core
  for (int c = warp; c < R; c += nwarp) {
    T best = (T)-1;
    int bidx = 0x7fffffff;
    for (int i = lane; i < s; i += 32) {
      const T v = fabs(Am[(long)i * R + c]);
      if (v > best || (v == best && i < bidx)) {
        best = v;
        bidx = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T ob = __shfl_xor_sync(kFull, best, o);
      const int oi = __shfl_xor_sync(kFull, bidx, o);
      if (ob > best || (ob == best && oi < bidx)) {
        best = ob;
        bidx = oi;
      }
    }
    if (lane == 0) sgn[c] = (bidx < s && Am[(long)bidx * R + c] < (T)0) ? (T)-1 : (T)1;
  }
  __syncthreads();
  for (int e = tid; e < s * R; e += nthr) {
    const int c = e - (e / R) * R;
    a.A_out[e] = sgn[c] * Am[e];
  }
  for (int e = tid; e < r * R; e += nthr) {
    const int rho = e / R, c = e - (e / R) * R;
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

template <typename T, typename U, bool POLISH64>
__global__ void __launch_bounds__(kThreads) k_lrls_fused(FusedArgs<T> a) {
  pdl_trigger();
  pdl_wait();
  lrls_fused_body<T, U, POLISH64>(a);
}

// Independent subproblems, one per block.
template <typename T, typename U, bool POLISH64>
__global__ void __launch_bounds__(kThreads) k_lrls_fused_batched(const FusedArgs<T>* __restrict__ args) {
  const FusedArgs<T> a = args[blockIdx.x];
  lrls_fused_body<T, U, POLISH64>(a);
}

// ---------------------------------------------------------------- host side

// Static shared memory of the kernel plus slack, kept out of the dynamic budget.
constexpr size_t kStaticReserve = 4096;

size_t lrls_fused_smem_bytes(int r, int s, int k, int R, int solve, size_t tsize, bool fp64,
                             bool* m_smem) {
  const bool polish = fp64 && tsize == 4;
  const size_t usz = (polish || tsize == 8) ? 8 : tsize;
  FusedLayout L = fused_layout(r, s, k, R, solve, tsize, usz, true, polish);
  bool on = true;
  if (L.total + kStaticReserve > kMaxSmem) {
    L = fused_layout(r, s, k, R, solve, tsize, usz, false, polish);
    on = false;
  }
  if (m_smem) *m_smem = on;
  return L.total + kStaticReserve;
}

bool lrls_fused_supported(int r, int s, int k, int R, int solve, size_t tsize, bool fp64) {
  if (r < 1 || s < 1 || R < 1 || k < R) return false;
  if (solve == TS_SOLVE_RSVD) {
    if (k > 32) return false;  // Householder: warp c owns column c
  } else if (r > kMaxEig) {
    return false;
  }
  return lrls_fused_smem_bytes(r, s, k, R, solve, tsize, fp64, nullptr) <= kMaxSmem;
}

template <typename T>
ts_status make_fused_args(int r, int s, int k, int R, int solve, bool fp64, const T* G, long ldg,
                          const T* W, long ldw, const T* H, long ldh, T* Mbuf, T* CnT, T* A_out,
                          T* core, CoreMap map, int* flag, FusedArgs<T>* out, size_t* smem) {
  if (!lrls_fused_supported(r, s, k, R, solve, sizeof(T), fp64))
    return fail(TS_ERR_SHAPE, "fused solve: r=%d s=%d k=%d R=%d does not fit one block", r, s, k,
                R);
  FusedArgs<T> a{};
  a.r = r;
  a.s = s;
  a.k = k;
  a.R = R;
  a.solve = solve;
  a.G = G;
  a.ldg = ldg;
  a.W = W;
  a.ldw = ldw;
  a.H = H;
  a.ldh = ldh;
  a.Mbuf = Mbuf;
  a.CnT = CnT;
  a.A_out = A_out;
  a.core = core;
  a.map = map;
  a.flag = flag;
  *smem = lrls_fused_smem_bytes(r, s, k, R, solve, sizeof(T), fp64, &a.m_smem) - kStaticReserve;
  *out = a;
  return TS_OK;
}

template <typename T>
ts_status launch_lrls_fused(int r, int s, int k, int R, int solve, bool fp64, const T* G,
                            long ldg, const T* W, long ldw, const T* H, long ldh, T* Mbuf, T* CnT,
                            T* A_out, T* core, CoreMap map, int* flag, cudaStream_t st) {
  if (lrls_chol_supported(r, s, k, R, solve, sizeof(T), fp64)) {
    FusedArgs<T> c{};
    c.r = r;
    c.s = s;
    c.k = k;
    c.R = R;
    c.solve = solve;
    c.G = G;
    c.ldg = ldg;
    c.W = W;
    c.ldw = ldw;
    c.H = H;
    c.ldh = ldh;
    c.Mbuf = Mbuf;
    c.CnT = CnT;
    c.A_out = A_out;
    c.core = core;
    c.map = map;
    c.flag = flag;
    return launch_lrls_chol<T>(c, fp64, st);
  }
  FusedArgs<T> a;
  size_t smem = 0;
  TS_TRY(make_fused_args<T>(r, s, k, R, solve, fp64, G, ldg, W, ldw, H, ldh, Mbuf, CnT, A_out,
                            core, map, flag, &a, &smem));
  const bool polish = fp64 && sizeof(T) == 4;
  if constexpr (sizeof(T) == 4) {
    if (polish) {
      TS_TRY(ensure_dynamic_smem((const void*)k_lrls_fused<T, double, true>, smem));
      return launch_pdl(k_lrls_fused<T, double, true>, dim3(1), dim3(kThreads), smem, st, a);
    }
  }
  TS_TRY(ensure_dynamic_smem((const void*)k_lrls_fused<T, T, false>, smem));
  return launch_pdl(k_lrls_fused<T, T, false>, dim3(1), dim3(kThreads), smem, st, a);
}

template <typename T>
ts_status launch_lrls_fused_batched(const FusedArgs<T>* args, int count, bool fp64, size_t smem,
                                    cudaStream_t st) {
  if (count < 1) return TS_OK;
  if constexpr (sizeof(T) == 4) {
    if (fp64) {
      TS_TRY(ensure_dynamic_smem((const void*)k_lrls_fused_batched<T, double, true>, smem));
      k_lrls_fused_batched<T, double, true><<<count, kThreads, smem, st>>>(args);
      TS_LAUNCH_CHECK();
      return TS_OK;
    }
  }
  TS_TRY(ensure_dynamic_smem((const void*)k_lrls_fused_batched<T, T, false>, smem));
  k_lrls_fused_batched<T, T, false><<<count, kThreads, smem, st>>>(args);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

#define TS_INST_FUSED(T)                                                                       \
  template ts_status make_fused_args<T>(int, int, int, int, int, bool, const T*, long, const T*, \
                                        long, const T*, long, T*, T*, T*, T*, CoreMap, int*,    \
                                        FusedArgs<T>*, size_t*);                                \
  template ts_status launch_lrls_fused_batched<T>(const FusedArgs<T>*, int, bool, size_t,       \
                                                  cudaStream_t);
TS_INST_FUSED(float)
TS_INST_FUSED(double)
#undef TS_INST_FUSED

template ts_status launch_lrls_fused<float>(int, int, int, int, int, bool, const float*, long,
                                            const float*, long, const float*, long, float*,
                                            float*, float*, float*, CoreMap, int*, cudaStream_t);
template ts_status launch_lrls_fused<double>(int, int, int, int, int, bool, const double*, long,
                                             const double*, long, const double*, long, double*,
                                             double*, double*, double*, CoreMap, int*,
                                             cudaStream_t);

}  // namespace ts
