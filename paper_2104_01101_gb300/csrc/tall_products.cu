// Products with one huge dimension s (a mode size of 10^5 and more) in the subproblems
// of Alg. 5, where the general tiled product wastes most of its tile on the narrow
// side:
//   D = M^T Y   (k x s):  M (m x k, k <= 32) tall, Y (m x s) wide.  One pass over Y,
//               the operand that dominates the bytes; each thread owns 4 columns and
//               keeps k sums per column in registers, M's rows broadcast from shared
//               memory.  Each output is one thread's sum in row order.
//   P = Y Om    (m x n):  Y (m x s) wide, Om (s x n, n <= 80) tall.  A 128 x 80 output
//               tile per block over a chunk of s (split over s across blocks), the
//               chunks' partial products summed in chunk order by a second kernel.
#include "internal.cuh"

namespace ts {

namespace {

template <typename T, int KM>
__global__ void __launch_bounds__(128) k_tall_tn(int m, int k, long s, const T* __restrict__ M,
                                                 long ldm, const T* __restrict__ Y, long ldy,
                                                 T* __restrict__ D, long ldd) {
  constexpr int RB = 64;  // rows of M staged per round
  __shared__ __align__(16) T sm[RB][KM];
  const long j0 = (long)blockIdx.x * 512 + threadIdx.x;
  T acc[4][KM];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int a = 0; a < KM; ++a) acc[q][a] = 0;
  for (int i0 = 0; i0 < m; i0 += RB) {
    const int ni = min(RB, m - i0);
    __syncthreads();
    for (int t = threadIdx.x; t < RB * KM; t += blockDim.x) {
      const int r = t / KM, a = t % KM;
      sm[r][a] = (r < ni && a < k) ? M[(long)(i0 + r) * ldm + a] : (T)0;
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < ni; ++r) {
      const T* yr = Y + (long)(i0 + r) * ldy;
      T y[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long j = j0 + q * 128;
        y[q] = j < s ? __ldcs(yr + j) : (T)0;  // streamed once: evict first
      }
#pragma unroll
      for (int a = 0; a < KM; ++a) {
        const T mv = sm[r][a];
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[q][a] += mv * y[q];
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const long j = j0 + q * 128;
    if (j < s)
#pragma unroll
      for (int a = 0; a < KM; ++a)
        if (a < k) D[(long)a * ldd + j] = acc[q][a];
  }
}

template <typename T>
struct WideTile {
  static constexpr int BM = 128, BN = 80, BK = sizeof(T) == 4 ? 32 : 16;
};

// Block (rt, c): rows [128 rt, 128 rt + 128) of P over s-chunk c, into part[c].
template <typename T>
__global__ void __launch_bounds__(256) k_wide_nn(int m, int n, long s, const T* __restrict__ Y,
                                                 long ldy, const T* __restrict__ Om, long ldo,
                                                 long chunk, T* __restrict__ part) {
  constexpr int BM = WideTile<T>::BM, BN = WideTile<T>::BN, BK = WideTile<T>::BK;
  __shared__ T ys[BK][BM + 1];  // Y tile, transposed (k-major): conflict-free both ways
  __shared__ T os[BK][BN];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads
  const int r0 = blockIdx.x * BM;
  const long k0 = (long)blockIdx.y * chunk;
  const long k1 = min(s, k0 + chunk);
  T acc[8][5];
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[u][v] = 0;
  for (long kk = k0; kk < k1; kk += BK) {
    // Y tile: BM rows x BK columns, lanes along the row (coalesced)
    for (int t = threadIdx.x; t < BM * BK; t += blockDim.x) {
      const int c = t % BK, r = t / BK;
      const long j = kk + c;
      ys[c][r] = (r0 + r < m && j < k1) ? __ldcs(Y + (long)(r0 + r) * ldy + j) : (T)0;
    }
    for (int t = threadIdx.x; t < BK * BN; t += blockDim.x) {
      const int c = t % BN, kr = t / BN;
      const long j = kk + kr;
      os[kr][c] = (c < n && j < k1) ? Om[j * ldo + c] : (T)0;
    }
    __syncthreads();
#pragma unroll 8
    for (int kr = 0; kr < BK; ++kr) {
      T y[8], o[5];
#pragma unroll
      for (int u = 0; u < 8; ++u) y[u] = ys[kr][ty + 16 * u];
#pragma unroll
      for (int v = 0; v < 5; ++v) o[v] = os[kr][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 5; ++v) acc[u][v] += y[u] * o[v];
    }
    __syncthreads();
  }
  T* out = part + (size_t)blockIdx.y * m * n;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int r = r0 + ty + 16 * u;
    if (r < m)
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        const int c = tx + 16 * v;
        if (c < n) out[(long)r * n + c] = acc[u][v];
      }
  }
}

// P(i, c) = sum over chunks z of part[z](i, c), in chunk order.
template <typename T>
__global__ void k_chunk_sum(int m, int n, int nsplit, const T* __restrict__ part,
                            T* __restrict__ P, long prs, long pcs) {
  const size_t mn = (size_t)m * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < mn;
       e += (size_t)gridDim.x * blockDim.x) {
    T v = 0;
    for (int z = 0; z < nsplit; ++z) v += part[z * mn + e];
    const long i = (long)(e / n), c = (long)(e % n);
    P[i * prs + c * pcs] = v;
  }
}

}  // namespace

template <typename T>
ts_status tall_tn(int m, int k, long s, const T* M, long ldm, const T* Y, long ldy, T* D,
                  long ldd, cudaStream_t st) {
  if (k < 1 || k > 32) return fail(TS_ERR_INVALID_ARG, "tall_tn: k=%d outside [1, 32]", k);
  const unsigned grid = (unsigned)((s + 511) / 512);
  if (k <= 16)
    k_tall_tn<T, 16><<<grid, 128, 0, st>>>(m, k, s, M, ldm, Y, ldy, D, ldd);
  else
    k_tall_tn<T, 32><<<grid, 128, 0, st>>>(m, k, s, M, ldm, Y, ldy, D, ldd);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

size_t wide_nn_partial_elems(int m, int n, long s) {
  const int rt = ceil_div(m, 128);
  const int nsplit = std::max(1, std::min(ceil_div(2 * 152, rt), ceil_div(s, 4096)));
  return (size_t)nsplit * m * std::min(n, 80);
}

template <typename T>
ts_status wide_nn(int m, int n, long s, const T* Y, long ldy, const T* Om, long ldo, T* P,
                  long prs, long pcs, T* part, size_t part_elems, cudaStream_t st) {
  const int rt = ceil_div(m, 128);
  const int nsplit = std::max(1, std::min(ceil_div(2 * 152, rt), ceil_div(s, 4096)));
  const long chunk = ((s + nsplit - 1) / nsplit + 31) / 32 * 32;
  for (int c0 = 0; c0 < n; c0 += 80) {
    const int nc = std::min(80, n - c0);
    if ((size_t)nsplit * m * nc > part_elems)
      return fail(TS_ERR_WORKSPACE, "wide_nn: partial buffer too small");
    k_wide_nn<T><<<dim3(rt, nsplit), 256, 0, st>>>(m, nc, s, Y, ldy, Om + c0, ldo, chunk, part);
    TS_LAUNCH_CHECK();
    const int blocks = std::max(1, std::min(ceil_div((long)m * nc, 256), 2048));
    k_chunk_sum<T><<<blocks, 256, 0, st>>>(m, nc, nsplit, part, P + c0 * pcs, prs, pcs);
    TS_LAUNCH_CHECK();
  }
  return TS_OK;
}

template ts_status tall_tn<float>(int, int, long, const float*, long, const float*, long, float*,
                                  long, cudaStream_t);
template ts_status tall_tn<double>(int, int, long, const double*, long, const double*, long,
                                   double*, long, cudaStream_t);
template ts_status wide_nn<float>(int, int, long, const float*, long, const float*, long, float*,
                                  long, long, float*, size_t, cudaStream_t);
template ts_status wide_nn<double>(int, int, long, const double*, long, const double*, long,
                                   double*, long, long, double*, size_t, cudaStream_t);

}  // namespace ts
