// Products with one huge dimension s (a mode size of 10^5 and more) in the subproblems
// of Alg. 5, where the general tiled product wastes most of its tile on the narrow
// side:
//   D = M^T Y   (k x s):  M (m x k, k <= 32) tall, Y (m x s) wide.  One pass over Y,
//               the operand that dominates the bytes; each thread owns two columns and
//               keeps their k sums in registers, M's rows broadcast from shared memory.
//               Each output is one thread's sum in row order.
//   K = D D^T   (k x k):  D (k x s) wide; a block per chunk of columns, partial
//               products summed in chunk order.
//   P = Y Om    (m x n):  Y (m x s) wide, Om (s x n) tall.  A 128 x 80 output tile (128 x
//               16 when n <= 16) per block over a chunk of s (split over s across
//               blocks), the chunks' partial products summed in chunk order afterwards.
#include "internal.cuh"

namespace ts {

namespace {

// Two columns of D per thread, 32 values of Y in flight per thread (enough bytes in
// flight to stream Y near HBM speed in a single wave of blocks).
template <typename T, int KM>
__global__ void __launch_bounds__(256) k_tall_tn(int m, int k, long s, const T* __restrict__ M,
                                                 long ldm, const T* __restrict__ Y, long ldy,
                                                 T* __restrict__ D, long ldd, int rows_per) {
  // rows [rows_per * blockIdx.y, +rows_per) of M and Y; with gridDim.y > 1 the block
  // writes its partial product to D + blockIdx.y * k * ldd (summed in order afterwards)
  const int ib = blockIdx.y * rows_per;
  M += (long)ib * ldm;
  Y += (long)ib * ldy;
  m = min(rows_per, m - ib);
  D += (long)blockIdx.y * k * ldd;
  constexpr int RB = 64;  // rows of M staged per round
  constexpr int U = 16;   // rows of Y loaded ahead
  __shared__ __align__(16) T sm[RB][KM];
  const long j = (long)blockIdx.x * 2 * blockDim.x + threadIdx.x;  // and j + blockDim.x
  const long j2 = j + blockDim.x;
  const bool in = j < s, in2 = j2 < s;
  T acc[KM], acc2[KM];
#pragma unroll
  for (int a = 0; a < KM; ++a) acc[a] = acc2[a] = 0;
  for (int i0 = 0; i0 < m; i0 += RB) {
    const int ni = min(RB, m - i0);
    __syncthreads();
    for (int t = threadIdx.x; t < RB * KM; t += blockDim.x) {
      const int r = t / KM, a = t % KM;
      sm[r][a] = (r < ni && a < k) ? M[(long)(i0 + r) * ldm + a] : (T)0;
    }
    __syncthreads();
    for (int r0 = 0; r0 < ni; r0 += U) {
      T y[U], y2[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const T* row = Y + (long)(i0 + r0 + u) * ldy;
        y[u] = (in && r0 + u < ni) ? __ldcs(row + j) : (T)0;
        y2[u] = (in2 && r0 + u < ni) ? __ldcs(row + j2) : (T)0;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int r = r0 + u;  // < RB; y[u] = y2[u] = 0 beyond ni
#pragma unroll
        for (int a = 0; a < KM; ++a) {
          acc[a] += sm[r][a] * y[u];
          acc2[a] += sm[r][a] * y2[u];
        }
      }
    }
  }
#pragma unroll
  for (int a = 0; a < KM; ++a)
    if (a < k) {
      if (in) D[(long)a * ldd + j] = acc[a];
      if (in2) D[(long)a * ldd + j2] = acc2[a];
    }
}

template <typename T, int BN_>
struct WideTile {
  static constexpr int BM = 128, BN = BN_, BK = sizeof(T) == 4 ? 32 : 16;
  static constexpr int TN = BN_ / 16;  // columns per thread (strided by 16)
};

// Block (rt, c): rows [128 rt, 128 rt + 128) of P over s-chunk c, into part[c].  The
// next tile's global loads are issued into registers before the current tile's products
// (one tile in flight while computing).
template <typename T, int BNW>
__global__ void __launch_bounds__(256) k_wide_nn(int m, int n, long s, const T* __restrict__ Y,
                                                 long ldy, const T* __restrict__ Om, long ldo,
                                                 long chunk, T* __restrict__ part) {
  constexpr int BM = WideTile<T, BNW>::BM, BN = WideTile<T, BNW>::BN, BK = WideTile<T, BNW>::BK;
  constexpr int TN = WideTile<T, BNW>::TN;
  constexpr int NY = BM * BK / 256, NO = BK * BN / 256;
  __shared__ __align__(16) T ys[BK][BM + 4];  // Y tile, transposed (k-major), 16-byte rows
  __shared__ T os[BK][BN];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads
  const int r0 = blockIdx.x * BM;
  const long k0 = (long)blockIdx.y * chunk;
  const long k1 = min(s, k0 + chunk);
  T acc[8][TN];
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < TN; ++v) acc[u][v] = 0;
  T yv[NY], ov[NO];
  auto fetch = [&](long kk) {
#pragma unroll
    for (int q = 0; q < NY; ++q) {  // lanes along a row of Y (coalesced)
      const int t = threadIdx.x + 256 * q;
      const int c = t % BK, r = t / BK;
      const long j = kk + c;
      yv[q] = (r0 + r < m && j < k1) ? __ldcs(Y + (long)(r0 + r) * ldy + j) : (T)0;
    }
#pragma unroll
    for (int q = 0; q < NO; ++q) {
      const int t = threadIdx.x + 256 * q;
      const int c = t % BN, kr = t / BN;
      const long j = kk + kr;
      ov[q] = (c < n && j < k1) ? Om[j * ldo + c] : (T)0;
    }
  };
  auto stage = [&]() {
#pragma unroll
    for (int q = 0; q < NY; ++q) {
      const int t = threadIdx.x + 256 * q;
      ys[t % BK][t / BK] = yv[q];
    }
#pragma unroll
    for (int q = 0; q < NO; ++q) {
      const int t = threadIdx.x + 256 * q;
      os[t / BN][t % BN] = ov[q];
    }
  };
  if (k0 < k1) fetch(k0);
  for (long kk = k0; kk < k1; kk += BK) {
    __syncthreads();  // the previous tile's products are done
    stage();
    __syncthreads();
    if (kk + BK < k1) fetch(kk + BK);
#pragma unroll 8
    for (int kr = 0; kr < BK; ++kr) {
      T y[8], o[TN];
#pragma unroll
      for (int u = 0; u < 8; ++u) y[u] = ys[kr][8 * ty + u];  // two 16-byte loads
#pragma unroll
      for (int v = 0; v < TN; ++v) o[v] = os[kr][tx + 16 * v];
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < TN; ++v) acc[u][v] += y[u] * o[v];
    }
  }
  T* out = part + (size_t)blockIdx.y * m * n;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int r = r0 + 8 * ty + u;
    if (r < m)
#pragma unroll
      for (int v = 0; v < TN; ++v) {
        const int c = tx + 16 * v;
        if (c < n) out[(long)r * n + c] = acc[u][v];
      }
  }
}

// Block b: the k x k products of D's rows over its chunk of columns, into part[b].
template <typename T>
__global__ void __launch_bounds__(256) k_gram_wide(int k, long s, const T* __restrict__ D,
                                                   long ldd, long chunk, T* __restrict__ part) {
  __shared__ T ds[32][257];  // padded rows: conflict-free column reads across rows
  const long c1 = min(s, (long)(blockIdx.x + 1) * chunk);
  T acc[4] = {0, 0, 0, 0};
  for (long c0 = (long)blockIdx.x * chunk; c0 < c1; c0 += 256) {
    const int nc = (int)min(256L, c1 - c0);
    __syncthreads();
    for (int a = 0; a < k; ++a)
      ds[a][threadIdx.x] = threadIdx.x < nc ? D[(long)a * ldd + c0 + threadIdx.x] : (T)0;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int p = threadIdx.x + 256 * q;
      if (p < k * k) {
        const int a = p / k, b = p % k;
        T v = 0;
        for (int t = 0; t < nc; ++t) v += ds[a][t] * ds[b][t];
        acc[q] += v;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int p = threadIdx.x + 256 * q;
    if (p < k * k) part[(long)blockIdx.x * k * k + p] = acc[q];
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

// Resident blocks of a kernel on the current device (cached per device; racing first
// calls compute the same value).
static int resident_blocks(const void* kernel, int threads, int* cache) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 16) dev = 0;
  if (cache[dev] == 0) {
    int nsm = 0, b = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, 0);
    cache[dev] = std::max(1, nsm * std::max(1, b));
  }
  return cache[dev];
}

template <typename T>
ts_status tall_tn(int m, int k, long s, const T* M, long ldm, const T* Y, long ldy, T* D,
                  long ldd, T* part, size_t part_elems, cudaStream_t st) {
  if (k < 1 || k > 32) return fail(TS_ERR_INVALID_ARG, "tall_tn: k=%d outside [1, 32]", k);
  const int tiles = (int)((s + 511) / 512);
  // rows split so that the blocks fill ~8 waves (a partial last wave then costs little)
  static int cache[16] = {};
  const int sl = resident_blocks((const void*)k_tall_tn<T, 16>, 256, cache);
  int ns = (8 * sl + tiles / 2) / tiles;
  ns = std::max(1, std::min(ns, std::min(32, m / 256)));
  while (ns > 1 && (size_t)ns * k * s > part_elems) --ns;
  const int rows_per = ceil_div(m, ns);
  ns = ceil_div(m, rows_per);
  T* out = ns > 1 ? part : D;
  const long ldo = ns > 1 ? s : ldd;
  const dim3 grid((unsigned)tiles, (unsigned)ns);
  if (k <= 16)
    k_tall_tn<T, 16><<<grid, 256, 0, st>>>(m, k, s, M, ldm, Y, ldy, out, ldo, rows_per);
  else
    k_tall_tn<T, 32><<<grid, 256, 0, st>>>(m, k, s, M, ldm, Y, ldy, out, ldo, rows_per);
  TS_LAUNCH_CHECK();
  if (ns > 1) {
    const int blocks = std::max(1, std::min(ceil_div((long)k * s, 256), 2048));
    k_chunk_sum<T><<<blocks, 256, 0, st>>>(k, (int)s, ns, part, D, ldd, 1);
    TS_LAUNCH_CHECK();
  }
  return TS_OK;
}

template <typename T>
ts_status gram_wide(int k, long s, const T* D, long ldd, T* K, long ldk, T* part,
                    size_t part_elems, cudaStream_t st) {
  if (k < 1 || k > 32) return fail(TS_ERR_INVALID_ARG, "gram_wide: k=%d outside [1, 32]", k);
  const int nb = (int)std::min<long>(2 * 152, (s + 1023) / 1024);
  const long chunk = (s + nb - 1) / nb;
  if ((size_t)nb * k * k > part_elems)
    return fail(TS_ERR_WORKSPACE, "gram_wide: partial buffer too small");
  k_gram_wide<T><<<nb, 256, 0, st>>>(k, s, D, ldd, chunk, part);
  TS_LAUNCH_CHECK();
  k_chunk_sum<T><<<1, 256, 0, st>>>(k, k, nb, part, K, ldk, 1);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

// Chunks of s per row tile: as many as fill one wave of resident blocks (a partial
// second wave would cost a whole block time), at least 4096 columns each.
template <typename T, int BNW>
static int wide_nn_splits(int m, long s) {
  static int cache[16] = {};
  const int b = resident_blocks((const void*)k_wide_nn<T, BNW>, 256, cache);
  const int rt = ceil_div(m, 128);
  return std::max(1, std::min(b / rt, ceil_div(s, 4096)));
}

template <typename T>
ts_status wide_nn(int m, int n, long s, const T* Y, long ldy, const T* Om, long ldo, T* P,
                  long prs, long pcs, T* part, size_t part_elems, cudaStream_t st) {
  const bool narrow = n <= 16;  // a 16-column tile: the 80-column one would idle 5/6 of it
  const int nsplit = narrow ? wide_nn_splits<T, 16>(m, s) : wide_nn_splits<T, 80>(m, s);
  const int rt = ceil_div(m, 128);
  const long chunk = ((s + nsplit - 1) / nsplit + 31) / 32 * 32;
  for (int c0 = 0; c0 < n; c0 += 80) {
    const int nc = std::min(80, n - c0);
    if ((size_t)nsplit * m * nc > part_elems)
      return fail(TS_ERR_WORKSPACE, "wide_nn: partial buffer too small");
    if (narrow)
      k_wide_nn<T, 16><<<dim3(rt, nsplit), 256, 0, st>>>(m, nc, s, Y, ldy, Om + c0, ldo, chunk,
                                                         part);
    else
      k_wide_nn<T, 80><<<dim3(rt, nsplit), 256, 0, st>>>(m, nc, s, Y, ldy, Om + c0, ldo, chunk,
                                                         part);
    TS_LAUNCH_CHECK();
    const int blocks = std::max(1, std::min(ceil_div((long)m * nc, 256), 2048));
    k_chunk_sum<T><<<blocks, 256, 0, st>>>(m, nc, nsplit, part, P + c0 * pcs, prs, pcs);
    TS_LAUNCH_CHECK();
  }
  return TS_OK;
}

template ts_status tall_tn<float>(int, int, long, const float*, long, const float*, long, float*,
                                  long, float*, size_t, cudaStream_t);
template ts_status tall_tn<double>(int, int, long, const double*, long, const double*, long,
                                   double*, long, double*, size_t, cudaStream_t);
template ts_status gram_wide<float>(int, long, const float*, long, float*, long, float*, size_t,
                                    cudaStream_t);
template ts_status gram_wide<double>(int, long, const double*, long, double*, long, double*,
                                     size_t, cudaStream_t);
template ts_status wide_nn<float>(int, int, long, const float*, long, const float*, long, float*,
                                  long, long, float*, size_t, cudaStream_t);
template ts_status wide_nn<double>(int, int, long, const double*, long, const double*, long,
                                   double*, long, long, double*, size_t, cudaStream_t);

}  // namespace ts
