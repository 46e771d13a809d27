// Device helpers shared by the one-block dense linear algebra kernels of the
// sketched subproblem (Sec. 4): warp reductions and the round-robin Jacobi sweep.
#pragma once

#include "internal.cuh"

namespace ts {

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

// ---------------------------------------------------------------- symmetric eigensolver

struct JacobiShape {
  int n;   // matrix order
  int np;  // n rounded up to even (round-robin players)
  int lg;  // log2 of the column stride (power of two >= n)
};

// Barrier policies: the whole block, or the first nthr threads (named barrier 1).
struct BlockSync {
  __device__ void operator()() const { __syncthreads(); }
  __device__ int size() const { return blockDim.x; }
};
struct SubSync {
  int nthr;  // multiple of 32
  __device__ void operator()() const { asm volatile("bar.sync 1, %0;" ::"r"(nthr) : "memory"); }
  __device__ int size() const { return nthr; }
};

// Threads the Jacobi sweep of a matrix of order n keeps busy (pairs x padded columns).
__host__ __device__ inline int jacobi_threads(int n) {
  int lg = 0;
  while ((1 << lg) < n) ++lg;
  const int work = (((n + 1) & ~1) / 2) << lg;
  int t = ((work + 31) / 32) * 32;
  return t < 64 ? 64 : (t > 512 ? 512 : t);
}

// One cyclic sweep with round-robin pairing on A (n x n, row stride n); V accumulates.
// Called by the threads of `sync` (threadIdx.x < sync.size()).
template <typename U, typename Sync = BlockSync>
__device__ void jacobi_sweep(U* A, U* V, const JacobiShape& js, int* rp, int* rq, U* rc, U* rs,
                             Sync sync = Sync()) {
  const int n = js.n, np = js.np, npairs = np / 2;
  const int np2 = 1 << js.lg;
  const int nthr = sync.size();
  for (int t = 0; t < np - 1; ++t) {
    if (threadIdx.x < npairs) {
      const int i = threadIdx.x;
      const int a = i == 0 ? t : (t + i) % (np - 1);
      const int b = i == 0 ? np - 1 : (t - i + np - 1) % (np - 1);
      int p = min(a, b);
      const int q = max(a, b);
      U c = 1, s = 0;
      if (q < n) {
        const U apq = A[p * n + q];
        if (apq != (U)0) {
          const U theta = (A[q * n + q] - A[p * n + p]) / (2 * apq);
          const U tt = (theta >= (U)0 ? (U)1 : (U)-1) / (fabs(theta) + sqrt(theta * theta + (U)1));
          c = (U)1 / sqrt(tt * tt + (U)1);
          s = tt * c;
        }
      } else {
        p = -1;
      }
      rp[i] = p;
      rq[i] = q;
      rc[i] = c;
      rs[i] = s;
    }
    sync();
    for (int e = threadIdx.x; e < npairs * np2; e += nthr) {  // rows p, q
      const int i = e >> js.lg, l = e & (np2 - 1);
      const int p = rp[i];
      if (p < 0 || l >= n) continue;
      const int q = rq[i];
      const U c = rc[i], s = rs[i];
      const U ap = A[p * n + l], aq = A[q * n + l];
      A[p * n + l] = c * ap - s * aq;
      A[q * n + l] = s * ap + c * aq;
    }
    sync();
    // columns p, q and V: consecutive threads take consecutive pairs of one row l (the
    // other order, a column per warp, hits one bank 32 times when n is a multiple of 32)
    for (int e = threadIdx.x; e < npairs * n; e += nthr) {
      const int i = e % npairs, l = e / npairs;
      const int p = rp[i];
      if (p < 0) continue;
      const int q = rq[i];
      const U c = rc[i], s = rs[i];
      const U ap = A[l * n + p], aq = A[l * n + q];
      A[l * n + p] = c * ap - s * aq;
      A[l * n + q] = s * ap + c * aq;
      const U vp = V[l * n + p], vq = V[l * n + q];
      V[l * n + p] = c * vp - s * vq;
      V[l * n + q] = s * vp + c * vq;
    }
    sync();
  }
}

// Off-diagonal and total squared Frobenius norms (valid in every participating thread;
// red holds 2 * (threads / 32) + 2 values).
template <typename U, typename Sync = BlockSync>
__device__ void jacobi_norms(const U* A, int n, U* red, U& off, U& tot, Sync sync = Sync()) {
  const int nthr = sync.size();
  U o = 0, a = 0;
  for (int e = threadIdx.x; e < n * n; e += nthr) {
    const U v = A[e];
    a += v * v;
    if (e / n != e % n) o += v * v;
  }
  o = warp_sum(o);
  a = warp_sum(a);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = nthr >> 5;
  if (lane == 0) {
    red[2 * warp] = o;
    red[2 * warp + 1] = a;
  }
  sync();
  if (threadIdx.x == 0) {
    U so = 0, sa = 0;
    for (int w = 0; w < nw; ++w) {
      so += red[2 * w];
      sa += red[2 * w + 1];
    }
    red[2 * nw] = so;
    red[2 * nw + 1] = sa;
  }
  sync();
  off = red[2 * nw];
  tot = red[2 * nw + 1];
  sync();
}

}  // namespace ts
