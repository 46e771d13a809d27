// Relative residual ||T - T~||_F / ||T||_F of a Tucker model against a dense
// tensor (Sec. 7 fitness f = 1 - residual), by direct reconstruction:
//   Q = C x_1 A^(1) ... x_{N-1} A^(N-1)   (all modes but the last, small)
//   T~(row, :) = Q(row, :) A^(N)T          (streamed against T, row by row)
// Squares are summed per row in the data type and across rows in FP64.
#include "internal.cuh"

namespace ts {

struct FitDesc {
  int order;
  int64_t dims[TS_MAX_ORDER];
  int ranks[TS_MAX_ORDER];
  const void* factors[TS_MAX_ORDER];
};

template <typename T>
__global__ void k_fit_partial(FitDesc d, const T* __restrict__ core, T* __restrict__ Q,
                              int64_t nrows) {
  const int N = d.order;
  const int Rl = d.ranks[N - 1];
  int nr = 1;
  for (int k = 0; k < N - 1; ++k) nr *= d.ranks[k];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nrows * Rl;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / Rl;
    const int rl = (int)(e % Rl);
    int64_t idx[TS_MAX_ORDER];
    int64_t x = row;
    for (int k = N - 2; k >= 0; --k) {
      idx[k] = x % d.dims[k];
      x /= d.dims[k];
    }
    T acc = 0;
    for (int t = 0; t < nr; ++t) {
      T prod = core[(int64_t)t * Rl + rl];
      int y = t;
      for (int k = N - 2; k >= 0; --k) {
        const int rk = y % d.ranks[k];
        y /= d.ranks[k];
        prod *= static_cast<const T*>(d.factors[k])[idx[k] * d.ranks[k] + rk];
      }
      acc += prod;
    }
    Q[e] = acc;
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One warp per row of T (rows are the last-mode fibres).  The last factor is
// staged transposed in shared memory when it fits (AT[r][j]).
template <typename T>
__global__ void __launch_bounds__(256) k_fit_stream(const T* __restrict__ X,
                                                    const T* __restrict__ Q,
                                                    const T* __restrict__ Alast, int64_t nrows,
                                                    int sl, int Rl, int staged,
                                                    double* __restrict__ acc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* qs = reinterpret_cast<T*>(smem_raw);  // 8 warps x Rl
  T* AT = qs + 8 * Rl;                      // Rl x sl when staged
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (staged)
    for (int e = threadIdx.x; e < sl * Rl; e += blockDim.x) {
      const int j = e / Rl, r = e % Rl;
      AT[r * sl + j] = Alast[e];
    }
  __syncthreads();
  double d2 = 0, t2 = 0;
  for (int64_t row = blockIdx.x * 8 + warp; row < nrows; row += (int64_t)gridDim.x * 8) {
    for (int r = lane; r < Rl; r += 32) qs[warp * Rl + r] = Q[row * Rl + r];
    __syncwarp();
    T pd = 0, pt = 0;
    for (int j = lane; j < sl; j += 32) {
      T t = 0;
      if (staged) {
        for (int r = 0; r < Rl; ++r) t += qs[warp * Rl + r] * AT[r * sl + j];
      } else {
        for (int r = 0; r < Rl; ++r) t += qs[warp * Rl + r] * Alast[(int64_t)j * Rl + r];
      }
      const T x = X[row * sl + j];
      const T df = x - t;
      pd += df * df;
      pt += x * x;
    }
    d2 += (double)pd;
    t2 += (double)pt;
    __syncwarp();
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

template <typename T>
size_t fit_dense_scratch_elems(const ts_tensor& X, const int* ranks) {
  int64_t nrows = 1;
  for (int k = 0; k < X.order - 1; ++k) nrows *= X.dims[k];
  return (size_t)nrows * ranks[X.order - 1];
}

template <typename T>
ts_status launch_fit_dense(const ts_tensor& X, const int* ranks, const T* core,
                           const T* const* factors, T* Q, double* acc, double* residual_out,
                           cudaStream_t st) {
  FitDesc d{};
  d.order = X.order;
  int64_t nrows = 1;
  for (int k = 0; k < X.order; ++k) {
    d.dims[k] = X.dims[k];
    d.ranks[k] = ranks[k];
    d.factors[k] = factors[k];
    if (k < X.order - 1) nrows *= X.dims[k];
  }
  const int N = X.order;
  const int Rl = ranks[N - 1];
  const int sl = (int)X.dims[N - 1];
  TS_CUDA(cudaMemsetAsync(acc, 0, 2 * sizeof(double), st));
  {
    int64_t tot = nrows * Rl;
    int blocks = (int)((tot + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_fit_partial<T><<<blocks, 256, 0, st>>>(d, core, Q, nrows);
    TS_LAUNCH_CHECK();
  }
  size_t smem = sizeof(T) * 8 * (size_t)Rl;
  const size_t stage_bytes = sizeof(T) * (size_t)Rl * sl;
  const int staged = (smem + stage_bytes) <= 160 * 1024 ? 1 : 0;
  if (staged) smem += stage_bytes;
  if (smem > 48 * 1024)
    TS_CUDA(cudaFuncSetAttribute((const void*)k_fit_stream<T>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int blocks = (int)((nrows + 7) / 8);
  if (blocks > 152 * 4) blocks = 152 * 4;
  k_fit_stream<T><<<blocks, 256, smem, st>>>(static_cast<const T*>(X.values), Q, factors[N - 1],
                                             nrows, sl, Rl, staged, acc);
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
