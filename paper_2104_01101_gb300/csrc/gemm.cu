// Small strided SIMT GEMM for the sketched-system products (Z^T Z, Z^T Y Omega,
// Z E, M^T Y, D D^T ...).  These are tall-skinny products of a few MFLOP each:
// the tile loop is latency-bound, so the design favours a deterministic split of
// the long dimension across many CTAs (partials reduced in a fixed order) over
// tensor-core tiles.
#include "internal.cuh"

namespace ts {

namespace {
constexpr int BM = 64, BN = 64, BK = 16, NT = 256;
}

template <typename T>
__global__ void __launch_bounds__(NT) k_gemm(int M, int N, int K, int kchunk, MatView<T> A,
                                             MatView<T> B, T alpha, T beta, OutView<T> C,
                                             T* __restrict__ partial) {
  __shared__ T As[BK][BM + 4];
  __shared__ T Bs[BK][BN + 4];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  const bool a_kfast = (A.cs == 1);
  const bool b_nfast = (B.cs == 1);
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0;
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
    for (int t = threadIdx.x; t < BM * BK; t += NT) {
      int i, kk;
      if (a_kfast) { i = t / BK; kk = t % BK; } else { kk = t / BM; i = t % BM; }
      const int gi = m0 + i, gk = k0 + kk;
      As[kk][i] = (gi < M && gk < kend) ? A.p[(long)gi * A.rs + (long)gk * A.cs] : (T)0;
    }
    for (int t = threadIdx.x; t < BN * BK; t += NT) {
      int j, kk;
      if (b_nfast) { kk = t / BN; j = t % BN; } else { j = t / BK; kk = t % BK; }
      const int gj = n0 + j, gk = k0 + kk;
      Bs[kk][j] = (gj < N && gk < kend) ? B.p[(long)gk * B.rs + (long)gj * B.cs] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = m0 + ty * 4 + i;
    if (gi >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = n0 + tx * 4 + j;
      if (gj >= N) continue;
      if (partial) {
        partial[(size_t)blockIdx.z * M * N + (size_t)gi * N + gj] = acc[i][j];
      } else {
        T* c = C.p + (long)gi * C.rs + (long)gj * C.cs;
        *c = beta == (T)0 ? alpha * acc[i][j] : alpha * acc[i][j] + beta * *c;
      }
    }
  }
}

template <typename T>
__global__ void k_gemm_reduce(int M, int N, int splits, const T* __restrict__ partial, T alpha,
                              T beta, OutView<T> C) {
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
ts_status gemm(int M, int N, int K, double alpha, MatView<T> A, MatView<T> B, double beta,
               OutView<T> C, T* partial, size_t partial_elems, cudaStream_t st) {
  if (M <= 0 || N <= 0) return TS_OK;
  const int tiles = ceil_div(M, BM) * ceil_div(N, BN);
  int splits = 1;
  if (partial && K > 4 * BK) {
    splits = 2 * 152 / tiles;
    if (splits < 1) splits = 1;
    splits = splits > ceil_div(K, 4 * BK) ? ceil_div(K, 4 * BK) : splits;
    if (splits > 64) splits = 64;
    const size_t cap = partial_elems / ((size_t)M * N);
    if ((size_t)splits > cap) splits = (int)cap;
    if (splits < 1) splits = 1;
  }
  int kchunk = ceil_div(ceil_div(K > 0 ? K : 1, splits), BK) * BK;
  splits = ceil_div(K > 0 ? K : 1, kchunk);
  dim3 grid(ceil_div(N, BN), ceil_div(M, BM), splits);
  if (splits == 1) {
    k_gemm<T><<<grid, NT, 0, st>>>(M, N, K, kchunk, A, B, (T)alpha, (T)beta, C, nullptr);
    TS_LAUNCH_CHECK();
  } else {
    k_gemm<T><<<grid, NT, 0, st>>>(M, N, K, kchunk, A, B, (T)alpha, (T)beta, C, partial);
    TS_LAUNCH_CHECK();
    const size_t MN = (size_t)M * N;
    int blocks = (int)((MN + 255) / 256);
    if (blocks > 1024) blocks = 1024;
    k_gemm_reduce<T><<<blocks, 256, 0, st>>>(M, N, splits, partial, (T)alpha, (T)beta, C);
    TS_LAUNCH_CHECK();
  }
  return TS_OK;
}

template ts_status gemm<float>(int, int, int, double, MatView<float>, MatView<float>, double,
                               OutView<float>, float*, size_t, cudaStream_t);
template ts_status gemm<double>(int, int, int, double, MatView<double>, MatView<double>, double,
                                OutView<double>, double*, size_t, cudaStream_t);

}  // namespace ts
