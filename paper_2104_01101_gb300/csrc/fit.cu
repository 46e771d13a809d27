// Relative residual ||T - T~||_F / ||T||_F of a Tucker model against a dense
// tensor (Sec. 7 fitness f = 1 - residual), by direct reconstruction:
//   Q = C x_1 A^(1) ... x_{N-1} A^(N-1)   (all modes but the last; successive TTMs)
//   T~(row, :) = Q(row, :) A^(N)T          (streamed against T, one pass)
// Squares are summed per thread in the data type, then in FP64 across threads.
#include "internal.cuh"

namespace ts {

// out = in x_k A (C order): in is (a x Rk x b), A is (sk x Rk), out is (a x sk x b).
template <typename T>
__global__ void k_ttm(long a, int Rk, long b, int sk, const T* __restrict__ in,
                      const T* __restrict__ A, T* __restrict__ out) {
  const long total = a * sk * b;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long y = e % b;
    const long xi = e / b;
    const int i = (int)(xi % sk);
    const long x = xi / sk;
    const T* src = in + x * Rk * b + y;
    const T* arow = A + (long)i * Rk;
    T acc = 0;
    for (int r = 0; r < Rk; ++r) acc += arow[r] * src[r * b];
    out[e] = acc;
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Register-tiled pass for R_last <= RMAX and s_last % 4 == 0: thread t of a block owns
// columns 4t..4t+3 of every row (their A^(N) rows live in registers); blocks stride over
// the rows.  T rows are read as float4/double2-pairs, coalesced.
template <typename T, int RMAX>
__global__ void __launch_bounds__(256) k_fit_stream_tiled(const T* __restrict__ X,
                                                          const T* __restrict__ Q,
                                                          const T* __restrict__ Alast,
                                                          int64_t nrows, int sl, int Rl,
                                                          double* __restrict__ acc) {
  const int nq = sl / 4;
  double d2 = 0, t2 = 0;
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    T a[4][RMAX];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int r = 0; r < RMAX; ++r) a[c][r] = r < Rl ? Alast[(long)(4 * q + c) * Rl + r] : (T)0;
    T pd = 0, pt = 0;
    // 4 rows of T in flight per thread (the read of T is the bound)
    const int64_t G = gridDim.x;
    for (int64_t row0 = blockIdx.x; row0 < nrows; row0 += 4 * G) {
      T xs[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t row = row0 + u * G;
        const T* xr = X + (row < nrows ? row : 0) * sl + 4 * q;
        if constexpr (sizeof(T) == 4) {
          const float4 v = __ldcs(reinterpret_cast<const float4*>(xr));
          xs[u][0] = v.x; xs[u][1] = v.y; xs[u][2] = v.z; xs[u][3] = v.w;
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c) xs[u][c] = xr[c];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t row = row0 + u * G;
        if (row >= nrows) break;
        T qr[RMAX];
#pragma unroll
        for (int r = 0; r < RMAX; ++r) qr[r] = r < Rl ? __ldg(&Q[row * Rl + r]) : (T)0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          T t = 0;
#pragma unroll
          for (int r = 0; r < RMAX; ++r) t += qr[r] * a[c][r];
          const T df = xs[u][c] - t;
          pd += df * df;
          pt += xs[u][c] * xs[u][c];
        }
      }
    }
    d2 += (double)pd;
    t2 += (double)pt;
  }
  d2 = warp_sum_d(d2);
  t2 = warp_sum_d(t2);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(acc, d2);
    atomicAdd(acc + 1, t2);
  }
}

// General pass: one warp per row, the last factor read from global memory.
template <typename T>
__global__ void __launch_bounds__(256) k_fit_stream(const T* __restrict__ X,
                                                    const T* __restrict__ Q,
                                                    const T* __restrict__ Alast, int64_t nrows,
                                                    int sl, int Rl, double* __restrict__ acc) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double d2 = 0, t2 = 0;
  for (int64_t row = blockIdx.x * 8 + warp; row < nrows; row += (int64_t)gridDim.x * 8) {
    T pd = 0, pt = 0;
    for (int j = lane; j < sl; j += 32) {
      T t = 0;
      for (int r = 0; r < Rl; ++r) t += Q[row * Rl + r] * Alast[(int64_t)j * Rl + r];
      const T x = X[row * sl + j];
      const T df = x - t;
      pd += df * df;
      pt += x * x;
    }
    d2 += (double)pd;
    t2 += (double)pt;
  }
  d2 = warp_sum_d(d2);
  t2 = warp_sum_d(t2);
  if (lane == 0) {
    atomicAdd(acc, d2);
    atomicAdd(acc + 1, t2);
  }
}

__global__ void k_fit_finish(const double* acc, double* out) {
  out[0] = acc[1] > 0 ? sqrt(acc[0] / acc[1]) : 0.0;
}

// Two buffers of |Q| = prod_{k < N-1} dims[k] * ranks[N-1] values each.
template <typename T>
size_t fit_dense_scratch_elems(const ts_tensor& X, const int* ranks) {
  int64_t nrows = 1;
  for (int k = 0; k < X.order - 1; ++k) nrows *= X.dims[k];
  return 2 * (size_t)nrows * ranks[X.order - 1];
}

static int grid_for(long n) {
  long b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

template <typename T>
ts_status launch_fit_dense(const ts_tensor& X, const int* ranks, const T* core,
                           const T* const* factors, T* scratch, double* acc, double* residual_out,
                           cudaStream_t st) {
  const int N = X.order;
  int64_t nrows = 1;
  for (int k = 0; k < N - 1; ++k) nrows *= X.dims[k];
  const int Rl = ranks[N - 1];
  const int sl = (int)X.dims[N - 1];
  T* buf[2] = {scratch, scratch + (size_t)nrows * Rl};
  TS_CUDA(cudaMemsetAsync(acc, 0, 2 * sizeof(double), st));
  // Q by successive TTMs of the core along modes N-2, ..., 0
  const T* cur = core;
  long shape[TS_MAX_ORDER];
  for (int k = 0; k < N; ++k) shape[k] = ranks[k];
  int which = 0;
  for (int k = N - 2; k >= 0; --k) {
    long a = 1, b = 1;
    for (int j = 0; j < k; ++j) a *= shape[j];
    for (int j = k + 1; j < N; ++j) b *= shape[j];
    T* out = buf[which];
    k_ttm<T><<<grid_for(a * X.dims[k] * b), 256, 0, st>>>(a, ranks[k], b, (int)X.dims[k], cur,
                                                           factors[k], out);
    TS_LAUNCH_CHECK();
    shape[k] = X.dims[k];
    cur = out;
    which ^= 1;
  }
  const int blocks = (int)(nrows < 152 * 8 ? nrows : 152 * 8);
  if (sl % 4 == 0 && Rl <= 16 && sl / 4 <= 1024 && ((uintptr_t)X.values & 15) == 0) {
    const int threads = ((sl / 4 + 31) / 32) * 32;
    if (Rl <= 8)
      k_fit_stream_tiled<T, 8><<<blocks, threads, 0, st>>>(static_cast<const T*>(X.values), cur,
                                                           factors[N - 1], nrows, sl, Rl, acc);
    else
      k_fit_stream_tiled<T, 16><<<blocks, threads, 0, st>>>(static_cast<const T*>(X.values), cur,
                                                            factors[N - 1], nrows, sl, Rl, acc);
  } else {
    int b2 = (int)((nrows + 7) / 8);
    if (b2 > 152 * 4) b2 = 152 * 4;
    k_fit_stream<T><<<b2, 256, 0, st>>>(static_cast<const T*>(X.values), cur, factors[N - 1],
                                        nrows, sl, Rl, acc);
  }
  TS_LAUNCH_CHECK();
  k_fit_finish<<<1, 1, 0, st>>>(acc, residual_out);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

template size_t fit_dense_scratch_elems<float>(const ts_tensor&, const int*);
template size_t fit_dense_scratch_elems<double>(const ts_tensor&, const int*);
template ts_status launch_fit_dense<float>(const ts_tensor&, const int*, const float*,
                                           const float* const*, float*, double*, double*,
                                           cudaStream_t);
template ts_status launch_fit_dense<double>(const ts_tensor&, const int*, const double*,
                                            const double* const*, double*, double*, double*,
                                            cudaStream_t);

}  // namespace ts
