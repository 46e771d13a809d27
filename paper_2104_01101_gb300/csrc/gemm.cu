// Small strided SIMT GEMM for the sketched-system products ([Z^T Z | Z^T Y Omega | Z^T Y],
// Y Omega, Z E, M^T Y, D D^T, the Init-RRF products ...).  These are tall-skinny
// products of a few to a hundred MFLOP, latency-bound at the sizes of the method, so
// the launcher picks the output tile (64x64 or 32x32) that comes closest to one wave of
// CTAs and then splits the long dimension; split partials are summed in split order by
// a second, fully parallel kernel, so results are deterministic.  Inside a CTA the next
// K tile is fetched into registers while the current one is multiplied from shared
// memory, so the global latency of a tile overlaps the arithmetic of the previous one.
// The B operand may be up to three strided views side by side (columns [0, n1) from
// B1, [n1, n2) from B2 and [n2, N) from B3), so that Z^T [Z | Y Omega | Y] is one
// product even though Z is stored column-major and the others row-major.
#include "internal.cuh"

namespace ts {

namespace {
constexpr int BK = 32, NT = 256;
}

// Element (gk, gj) of the three-view B operand (zero outside [0, K) x [0, N)).
template <typename T>
__device__ __forceinline__ T b_at(const MatView<T>& B1, int n1, const MatView<T>& B2, int n2,
                                  const MatView<T>& B3, int N, int kend, int gk, int gj) {
  if (gj >= N || gk >= kend) return (T)0;
  if (gj < n1) return B1.p[(long)gk * B1.rs + (long)gj * B1.cs];
  if (gj < n2) return B2.p[(long)gk * B2.rs + (long)(gj - n1) * B2.cs];
  return B3.p[(long)gk * B3.rs + (long)(gj - n2) * B3.cs];
}

// C tile BM x BN over K range [kbeg, kend) of this split.  256 threads as 16 x 16, each
// owning a TM x TN register tile; As and Bs hold the current K tile (k-major rows).
template <typename T, int BM, int BN>
__device__ __forceinline__ void gemm_tile(int M, int N, int K, int kchunk, const MatView<T>& A,
                                          const MatView<T>& B1, int n1, const MatView<T>& B2,
                                          int n2, const MatView<T>& B3, T alpha, T beta,
                                          const OutView<T>& C, T* __restrict__ partial, int bx,
                                          int by, int bz) {
  constexpr int TM = BM / 16, TN = BN / 16;         // outputs per thread: TM x TN
  constexpr int LA = BM * BK / NT, LB = BN * BK / NT;  // tile elements each thread fetches
  __shared__ __align__(16) T As[BK][BM + 4];
  __shared__ __align__(16) T Bs[BK][BN + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = by * BM, n0 = bx * BN;
  const int kbeg = bz * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const bool a_kfast = (A.cs == 1);
  const MatView<T>& Bv = n0 < n1 ? B1 : (n0 < n2 ? B2 : B3);  // view this tile starts in
  const bool b_kfast = (Bv.rs == 1 && Bv.cs != 1);
  // fetch mapping (coalesced along the view's contiguous index)
  auto a_idx = [&](int t, int& i, int& kk) {
    if (a_kfast) { i = t / BK; kk = t % BK; } else { kk = t / BM; i = t % BM; }
  };
  auto b_idx = [&](int t, int& j, int& kk) {
    if (b_kfast) { j = t / BK; kk = t % BK; } else { kk = t / BN; j = t % BN; }
  };
  T ra[LA], rb[LB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int u = 0; u < LA; ++u) {
      int i, kk;
      a_idx(threadIdx.x + u * NT, i, kk);
      const int gi = m0 + i, gk = k0 + kk;
      ra[u] = (gi < M && gk < kend) ? A.p[(long)gi * A.rs + (long)gk * A.cs] : (T)0;
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      int j, kk;
      b_idx(threadIdx.x + u * NT, j, kk);
      rb[u] = b_at<T>(B1, n1, B2, n2, B3, N, kend, k0 + kk, n0 + j);
    }
  };
  auto stage = [&]() {
#pragma unroll
    for (int u = 0; u < LA; ++u) {
      int i, kk;
      a_idx(threadIdx.x + u * NT, i, kk);
      As[kk][i] = ra[u];
    }
#pragma unroll
    for (int u = 0; u < LB; ++u) {
      int j, kk;
      b_idx(threadIdx.x + u * NT, j, kk);
      Bs[kk][j] = rb[u];
    }
  };
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0;
  if (kbeg < kend) {
    fetch(kbeg);
    stage();
    __syncthreads();
  }
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    const bool more = k0 + BK < kend;
    if (more) fetch(k0 + BK);  // in flight during the products below
#pragma unroll 8
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
    if (more) {
      stage();
      __syncthreads();
    }
  }
  const size_t MN = (size_t)M * N;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gi = m0 + ty * TM + i;
    if (gi >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gj = n0 + tx * TN + j;
      if (gj >= N) continue;
      if (partial) {
        partial[bz * MN + (size_t)gi * N + gj] = acc[i][j];
      } else {
        T* c = C.p + (long)gi * C.rs + (long)gj * C.cs;
        *c = beta == (T)0 ? alpha * acc[i][j] : alpha * acc[i][j] + beta * *c;
      }
    }
  }
}

template <typename T, int BM, int BN>
__global__ void __launch_bounds__(NT) k_gemm(int M, int N, int K, int kchunk, MatView<T> A,
                                             MatView<T> B1, int n1, MatView<T> B2, int n2,
                                             MatView<T> B3, T alpha, T beta, OutView<T> C,
                                             T* __restrict__ partial, const int* skip) {
  pdl_trigger();
  pdl_wait();
  if (skip && *skip) return;
  gemm_tile<T, BM, BN>(M, N, K, kchunk, A, B1, n1, B2, n2, B3, alpha, beta, C, partial,
                       blockIdx.x, blockIdx.y, blockIdx.z);
}

// Independent products, one per blockIdx.z, each C = A [B1 | B2 | B3] (no split).
template <typename T, int BM, int BN>
__global__ void __launch_bounds__(NT) k_gemm_batched(const GemmJob<T>* __restrict__ jobs) {
  const GemmJob<T>& j = jobs[blockIdx.z];
  if ((int)blockIdx.x * BN >= j.N || (int)blockIdx.y * BM >= j.M) return;
  gemm_tile<T, BM, BN>(j.M, j.N, j.K, ((j.K + BK - 1) / BK) * BK, j.A, j.B1, j.n1, j.B2, j.n2,
                       j.B3, (T)1, (T)0, j.C, nullptr, blockIdx.x, blockIdx.y, 0);
}

template <typename T>
ts_status launch_gemm_batched(const GemmJob<T>* jobs, int count, int maxM, int maxN, int tile,
                              cudaStream_t st) {
  if (count < 1 || maxM < 1 || maxN < 1) return TS_OK;
  if (tile == 32)
    k_gemm_batched<T, 32, 32><<<dim3(ceil_div(maxN, 32), ceil_div(maxM, 32), count), NT, 0, st>>>(jobs);
  else
    k_gemm_batched<T, 64, 64><<<dim3(ceil_div(maxN, 64), ceil_div(maxM, 64), count), NT, 0, st>>>(jobs);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

template <typename T>
__global__ void k_gemm_reduce(int M, int N, int splits, const T* __restrict__ partial, T alpha,
                              T beta, OutView<T> C, const int* skip) {
  pdl_trigger();
  pdl_wait();
  if (skip && *skip) return;
  const size_t MN = (size_t)M * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < MN;
       e += (size_t)gridDim.x * blockDim.x) {
    T s = 0;
    for (int z = 0; z < splits; ++z) s += partial[z * MN + e];
    const int i = (int)(e / N), j = (int)(e % N);
    T* c = C.p + (long)i * C.rs + (long)j * C.cs;
    *c = beta == (T)0 ? alpha * s : alpha * s + beta * *c;
  }
}

template <typename T>
ts_status gemm3(int M, int N, int K, double alpha, MatView<T> A, MatView<T> B1, int n1,
                MatView<T> B2, int n2, MatView<T> B3, double beta, OutView<T> C,
                const GemmSplit<T>* split, cudaStream_t st) {
  if (M <= 0 || N <= 0) return TS_OK;
  constexpr int kWave = 2 * 152;  // two resident CTAs per SM: 4 warps per sub-partition
  const int tiles64 = ceil_div(M, 64) * ceil_div(N, 64);
  const int tiles32 = ceil_div(M, 32) * ceil_div(N, 32);
  // 64x64 tiles (twice the FMAs per shared-memory load) when they alone, or split along
  // K, can give every SM a CTA; else 32x32
  const bool small = tiles64 * ceil_div(K > 0 ? K : 1, 4 * BK) < kWave / 2;
  const int tiles = small ? tiles32 : tiles64;
  const int bm = small ? 32 : 64;
  int splits = 1;
  if (split && split->partial && tiles < kWave && K > 4 * BK) {
    splits = ceil_div(kWave, tiles);
    if (splits > ceil_div(K, 4 * BK)) splits = ceil_div(K, 4 * BK);
    if (splits > 32) splits = 32;
    const size_t cap = split->partial_elems / ((size_t)M * N);
    if ((size_t)splits > cap) splits = (int)cap;
    if (splits < 1) splits = 1;
  }
  const int kchunk = ceil_div(ceil_div(K > 0 ? K : 1, splits), BK) * BK;
  splits = ceil_div(K > 0 ? K : 1, kchunk);
  dim3 grid(ceil_div(N, bm), ceil_div(M, bm), splits);
  T* part = splits > 1 ? split->partial : nullptr;
  const int* skip = split ? split->skip : nullptr;
  if (small)
    TS_TRY(launch_pdl(k_gemm<T, 32, 32>, grid, dim3(NT), 0, st, M, N, K, kchunk, A, B1, n1, B2,
                      n2, B3, (T)alpha, (T)beta, C, part, skip));
  else
    TS_TRY(launch_pdl(k_gemm<T, 64, 64>, grid, dim3(NT), 0, st, M, N, K, kchunk, A, B1, n1, B2,
                      n2, B3, (T)alpha, (T)beta, C, part, skip));
  if (splits > 1) {
    const size_t MN = (size_t)M * N;
    int blocks = (int)((MN + 255) / 256);
    if (blocks > 2048) blocks = 2048;
    TS_TRY(launch_pdl(k_gemm_reduce<T>, dim3(blocks), dim3(256), 0, st, M, N, splits,
                      static_cast<const T*>(part), (T)alpha, (T)beta, C, skip));
  }
  return TS_OK;
}

template <typename T>
ts_status launch_split_reduce(int M, int N, int splits, const T* partial, T* C, long ldc,
                              cudaStream_t st) {
  const size_t MN = (size_t)M * N;
  int blocks = (int)((MN + 255) / 256);
  if (blocks > 2048) blocks = 2048;
  return launch_pdl(k_gemm_reduce<T>, dim3(blocks), dim3(256), 0, st, M, N, splits, partial, (T)1,
                    (T)0, OutView<T>{C, ldc, 1}, (const int*)nullptr);
}

template <typename T>
ts_status gemm2(int M, int N, int K, double alpha, MatView<T> A, MatView<T> B1, int n1,
                MatView<T> B2, double beta, OutView<T> C, const GemmSplit<T>* split,
                cudaStream_t st) {
  return gemm3<T>(M, N, K, alpha, A, B1, n1, B2, N, B2, beta, C, split, st);
}

template <typename T>
ts_status gemm(int M, int N, int K, double alpha, MatView<T> A, MatView<T> B, double beta,
               OutView<T> C, const GemmSplit<T>* split, cudaStream_t st) {
  return gemm3<T>(M, N, K, alpha, A, B, N, B, N, B, beta, C, split, st);
}

#define TS_INST(T)                                                                              \
  template ts_status gemm<T>(int, int, int, double, MatView<T>, MatView<T>, double, OutView<T>, \
                             const GemmSplit<T>*, cudaStream_t);                                \
  template ts_status gemm2<T>(int, int, int, double, MatView<T>, MatView<T>, int, MatView<T>,   \
                              double, OutView<T>, const GemmSplit<T>*, cudaStream_t);           \
  template ts_status launch_split_reduce<T>(int, int, int, const T*, T*, long, cudaStream_t);    \
  template ts_status launch_gemm_batched<T>(const GemmJob<T>*, int, int, int, int, cudaStream_t); \
  template ts_status gemm3<T>(int, int, int, double, MatView<T>, MatView<T>, int, MatView<T>,   \
                              int, MatView<T>, double, OutView<T>, const GemmSplit<T>*,         \
                              cudaStream_t);
TS_INST(float)
TS_INST(double)
#undef TS_INST

}  // namespace ts
