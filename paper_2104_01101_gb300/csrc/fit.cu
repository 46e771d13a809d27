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

// ---------------------------------------------------------------- streamed form
//
// The register-tiled pass above keeps only a few rows of T in flight per thread, and its
// loads wait behind the arithmetic of the rows before them (about 1.4 TB/s on the 400^3
// workload).  This form (FP32, s_last % 4 = 0, s_last <= 512, R_last <= 16, whole
// 4-row groups) streams the rows through a ring of shared-memory stages by 1-D bulk
// copies: 16 rows of T and the same 16 rows of Q per stage, one copy each (contiguous),
// full / empty mbarriers with time-bounded waits.  One producer warp; 16 consumer warps in
// four groups of four, a group taking rows g, g + 4, g + 8, g + 12 of every stage, each
// of its threads four columns, whose rows of A^(N) stay in registers.  An expired wait
// makes the residual NaN.

namespace {
constexpr int kFitRows = 16;                 // rows of T per stage
constexpr int kFitWarps = 16;                // consumer warps
constexpr int kFitThreads = 32 * (kFitWarps + 1);
constexpr int kFitStages = 6;
constexpr unsigned long long kFitWaitNs = 200ull * 1000 * 1000;  // 200 ms per wait

__device__ __forceinline__ unsigned fit_smem(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ bool fit_try(unsigned mbar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of the given parity; false after kFitWaitNs.
__device__ __forceinline__ bool fit_wait(unsigned mbar, unsigned parity) {
  if (fit_try(mbar, parity)) return true;
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  while (!fit_try(mbar, parity)) {
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > kFitWaitNs) return false;
  }
  return true;
}
__device__ __forceinline__ void fit_load(unsigned dst, const void* src, unsigned bytes,
                                         unsigned mbar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(mbar)
      : "memory");
}
}  // namespace

template <int RMAX>
__global__ void __launch_bounds__(kFitThreads, 1)
    k_fit_rows(const float* __restrict__ X, const float* __restrict__ Q,
               const float* __restrict__ Alast, int64_t nrows, int sl, int Rl,
               double* __restrict__ acc) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long full_bar[kFitStages], empty_bar[kFitStages];
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const size_t xbytes = (size_t)kFitRows * sl * 4, qbytes = (size_t)kFitRows * Rl * 4;
  const size_t stage_bytes = (xbytes + qbytes + 15) & ~(size_t)15;
  // this CTA's rows: whole stages, contiguous
  const int64_t nst = (nrows + kFitRows - 1) / kFitRows;
  const int64_t per = (nst + gridDim.x - 1) / gridDim.x;
  const int64_t s0 = (int64_t)blockIdx.x * per, s1 = min(nst, s0 + per);
  if (tid == 0) {
    abort_flag = 0;
    for (int st = 0; st < kFitStages; ++st) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(fit_smem(&full_bar[st])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(fit_smem(&empty_bar[st])),
                   "r"(kFitWarps)
                   : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (s1 <= s0) return;
  if (warp == kFitWarps) {
    // ---------------- producer
    if (lane == 0) {
      int64_t issued = s0;
      int st = 0, ph = 0;
      for (int64_t sg = s0; sg < s1; ++sg) {
        if (sg - s0 >= kFitStages &&
            !fit_wait(fit_smem(&empty_bar[st]), (unsigned)(ph ^ 1))) {
          atomicExch(&abort_flag, 1);
          break;
        }
        const int64_t r0 = sg * kFitRows;
        const int nr = (int)min((int64_t)kFitRows, nrows - r0);
        const unsigned bx = (unsigned)nr * sl * 4, bq = (unsigned)nr * Rl * 4;
        const unsigned mbar = fit_smem(&full_bar[st]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar),
                     "r"(bx + bq)
                     : "memory");
        unsigned char* sp = smem_raw + (size_t)st * stage_bytes;
        fit_load(fit_smem(sp), X + r0 * sl, bx, mbar);
        fit_load(fit_smem(sp + xbytes), Q + r0 * Rl, bq, mbar);
        issued = sg + 1;
        if (++st == kFitStages) {
          st = 0;
          ph ^= 1;
        }
      }
      // the copies in flight land before the block exits
      for (int64_t sg = max(s0, issued - kFitStages); sg < issued; ++sg)
        fit_wait(fit_smem(&full_bar[(int)((sg - s0) % kFitStages)]),
                 (unsigned)(((sg - s0) / kFitStages) & 1));
    }
  } else {
    // ---------------- consumers: group g (4 warps) takes rows g, g + 4, ... of a stage;
    // thread t of the group owns columns 4 t .. 4 t + 3
    const int g = warp >> 2, t = tid & 127;
    const bool cols = 4 * t < sl;
    float a[4][RMAX];
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int r = 0; r < RMAX; ++r)
        a[c][r] = (cols && r < Rl) ? Alast[(int64_t)(4 * t + c) * Rl + r] : 0.f;
    float pd = 0.f, pt = 0.f;
    bool aborted = false;
    int st = 0, ph = 0;
    for (int64_t sg = s0; sg < s1; ++sg) {
      if (!aborted) {
        aborted = *(volatile int*)&abort_flag != 0;
        if (!aborted && !fit_wait(fit_smem(&full_bar[st]), (unsigned)ph)) {
          atomicExch(&abort_flag, 1);
          aborted = true;
        }
      }
      if (!aborted) {
        const unsigned char* sp = smem_raw + (size_t)st * stage_bytes;
        const float* xs = reinterpret_cast<const float*>(sp);
        const float* qs = reinterpret_cast<const float*>(sp + xbytes);
        const int nr = (int)min((int64_t)kFitRows, nrows - sg * kFitRows);
#pragma unroll
        for (int u = 0; u < kFitRows / 4; ++u) {
          const int row = g + 4 * u;
          if (row < nr && cols) {
            float q[RMAX];
#pragma unroll
            for (int r = 0; r < RMAX; ++r) q[r] = r < Rl ? qs[row * Rl + r] : 0.f;
            const float4 x = *reinterpret_cast<const float4*>(xs + (size_t)row * sl + 4 * t);
            const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              float tv = 0.f;
#pragma unroll
              for (int r = 0; r < RMAX; ++r) tv = fmaf(q[r], a[c][r], tv);
              const float df = xv[c] - tv;
              pd = fmaf(df, df, pd);
              pt = fmaf(xv[c], xv[c], pt);
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(fit_smem(&empty_bar[st])) : "memory");
      if (++st == kFitStages) {
        st = 0;
        ph ^= 1;
      }
    }
    double d2 = warp_sum_d((double)pd), t2 = warp_sum_d((double)pt);
    if (lane == 0) {
      atomicAdd(acc, d2);
      atomicAdd(acc + 1, t2);
    }
  }
  __syncthreads();
  // an expired wait leaves the sums incomplete: the residual becomes NaN, not a wrong value
  if (tid == 0 && abort_flag) atomicAdd(acc, __longlong_as_double(0x7ff8000000000000ll));
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
  if (sizeof(T) == 4 && sl % 4 == 0 && sl <= 512 && Rl <= 16 && nrows % 4 == 0 &&
      ((uintptr_t)X.values & 15) == 0 && ((uintptr_t)cur & 15) == 0) {
    // the streamed form (see above)
    const size_t stage = ((size_t)kFitRows * (sl + Rl) * 4 + 15) & ~(size_t)15;
    const size_t smem = kFitStages * stage;
    int dev = 0, nsm = 0;
    TS_CUDA(cudaGetDevice(&dev));
    TS_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int64_t nst = (nrows + kFitRows - 1) / kFitRows;
    const int grid = (int)(nst < nsm ? nst : nsm);
    const float* Xf = reinterpret_cast<const float*>(X.values);
    const float* Qf = reinterpret_cast<const float*>(cur);
    const float* Af = reinterpret_cast<const float*>(factors[N - 1]);
    if (Rl <= 8) {
      TS_TRY(ensure_dynamic_smem((const void*)k_fit_rows<8>, smem));
      k_fit_rows<8><<<grid, kFitThreads, smem, st>>>(Xf, Qf, Af, nrows, sl, Rl, acc);
    } else if (Rl <= 12) {
      TS_TRY(ensure_dynamic_smem((const void*)k_fit_rows<12>, smem));
      k_fit_rows<12><<<grid, kFitThreads, smem, st>>>(Xf, Qf, Af, nrows, sl, Rl, acc);
    } else {
      TS_TRY(ensure_dynamic_smem((const void*)k_fit_rows<16>, smem));
      k_fit_rows<16><<<grid, kFitThreads, smem, st>>>(Xf, Qf, Af, nrows, sl, Rl, acc);
    }
  } else if (sl % 4 == 0 && Rl <= 16 && sl / 4 <= 1024 && ((uintptr_t)X.values & 15) == 0) {
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
