// Fibre index of a COO tensor for one mode n.  Leverage-score sampling (Sec. 3.2)
// picks m columns of the unfolding T_(n), i.e. m mode-n fibres addressed by the other
// coordinates (i_k)_{k != n}; the paper's cost analysis (Sec. 6) counts O(m s) for
// gathering them, which needs the nonzeros grouped by fibre.  The index is an
// open-addressing hash table (linear probing, capacity a power of two >= 2 nnz) keyed
// by the C-order linear index of (i_k)_{k != n}; occupied slot h owns the nonzeros
// beg[h] .. beg[h+1]-1 of the fibre (their mode-n coordinate and value).
//
// Build (once per tensor and mode): insert every key and count its nonzeros (CAS on
// the key), exclusive scan of the counts over the slots, then place every nonzero at
// beg[slot] + a per-slot cursor.  Nonzeros of one fibre keep no particular order;
// repeated coordinates are added by the gather, so only the rounding of their sum
// depends on that order.
#include "internal.cuh"

namespace ts {

namespace {

constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kScanThreads = 256;
constexpr int kScanPer = 16;
constexpr int kScanChunk = kScanThreads * kScanPer;

__device__ __forceinline__ unsigned long long fibre_key(const int32_t* __restrict__ idx,
                                                        int64_t nnz, int64_t e,
                                                        const FibreIndex& F) {
  unsigned long long key = 0;
  for (int k = 0; k < F.order; ++k)
    if (k != F.mode) key += (unsigned long long)idx[(int64_t)k * nnz + e] * F.stride[k];
  return key;
}

__global__ void k_fib_insert(const int32_t* __restrict__ idx, int64_t nnz, FibreIndex F,
                             int32_t* __restrict__ eslot, int* flag) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long key = fibre_key(idx, nnz, e, F);
    uint64_t h = mix64(key) & F.mask;
    bool placed = false;
    for (uint64_t p = 0; p <= F.mask; ++p) {
      // keys are written once: a non-empty value read here is final, an empty one is
      // confirmed (or replaced) by the CAS
      unsigned long long cur = __ldcg(F.keys + h);
      if (cur == kEmptyKey) cur = atomicCAS(F.keys + h, kEmptyKey, key);
      if (cur == kEmptyKey || cur == key) {
        if (eslot) eslot[e] = (int32_t)h;  // keys only: the slot of every nonzero
        else atomicAdd(F.cur + h, 1);
        placed = true;
        break;
      }
      h = (h + 1) & F.mask;
    }
    if (!placed && flag) atomicExch(flag, 2);  // full table: excluded by the capacity
  }
}

__device__ __forceinline__ int block_excl_scan_i32(int v, int* warp_tot, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) warp_tot[lane] = t;
  }
  __syncthreads();
  const int base = warp ? warp_tot[warp - 1] : 0;
  *total = warp_tot[nw - 1];
  __syncthreads();
  return base + x - v;
}

// part[b] = sum of cnt over chunk b
__global__ void __launch_bounds__(kScanThreads) k_scan_partials(const int32_t* __restrict__ cnt,
                                                                int64_t n, int32_t* part) {
  __shared__ int wt[32];
  const int64_t c0 = blockIdx.x * (int64_t)kScanChunk + (int64_t)threadIdx.x * kScanPer;
  int s = 0;
#pragma unroll
  for (int i = 0; i < kScanPer; ++i)
    if (c0 + i < n) s += cnt[c0 + i];
  int tot;
  block_excl_scan_i32(s, wt, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// exclusive scan of part[0..nb) in place, part[nb] = total; one block
__global__ void __launch_bounds__(1024) k_scan_top(int32_t* part, int64_t nb) {
  __shared__ int wt[32];
  const int64_t per = (nb + blockDim.x - 1) / blockDim.x;
  const int64_t a = threadIdx.x * per;
  int s = 0;
  for (int64_t i = a; i < a + per && i < nb; ++i) s += part[i];
  int tot;
  int run = block_excl_scan_i32(s, wt, &tot);
  for (int64_t i = a; i < a + per && i < nb; ++i) {
    const int v = part[i];
    part[i] = run;
    run += v;
  }
  if (threadIdx.x == 0) part[nb] = tot;
}

// beg[i] = exclusive prefix sum of cnt, beg[n] = total
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int32_t* __restrict__ cnt,
                                                             int64_t n, const int32_t* part,
                                                             int64_t nb, int32_t* beg) {
  __shared__ int wt[32];
  const int64_t c0 = blockIdx.x * (int64_t)kScanChunk + (int64_t)threadIdx.x * kScanPer;
  int v[kScanPer];
  int s = 0;
#pragma unroll
  for (int i = 0; i < kScanPer; ++i) {
    v[i] = c0 + i < n ? cnt[c0 + i] : 0;
    s += v[i];
  }
  int tot;
  int run = part[blockIdx.x] + block_excl_scan_i32(s, wt, &tot);
#pragma unroll
  for (int i = 0; i < kScanPer; ++i)
    if (c0 + i < n) {
      beg[c0 + i] = run;
      run += v[i];
    }
  if (blockIdx.x == 0 && threadIdx.x == 0) beg[n] = part[nb];
}

template <typename T>
__global__ void k_fib_fill(const int32_t* __restrict__ idx, const T* __restrict__ vals,
                           int64_t nnz, FibreIndex F, int* flag) {
  T* val = static_cast<T*>(F.val);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long key = fibre_key(idx, nnz, e, F);
    uint64_t h = mix64(key) & F.mask;
    bool placed = false;
    for (uint64_t p = 0; p <= F.mask; ++p) {
      const unsigned long long cur = __ldg(F.keys + h);
      if (cur == key) {
        const int q = F.beg[h] + atomicAdd(F.cur + h, 1);
        F.pos[q] = idx[(int64_t)F.mode * nnz + e];
        val[q] = vals[e];
        placed = true;
        break;
      }
      if (cur == kEmptyKey) break;
      h = (h + 1) & F.mask;
    }
    if (!placed && flag) atomicExch(flag, 2);
  }
}

}  // namespace

int64_t fibre_index_capacity(int64_t nnz) {
  int64_t cap = 256;
  while (cap < 2 * nnz) cap <<= 1;
  return cap;
}

bool fibre_keys_fit(const ts_tensor& X, int mode) {
  // the linear index of (i_k)_{k != n} and the empty marker must fit 64 bits
  double c = 1;
  for (int k = 0; k < X.order; ++k)
    if (k != mode) c *= (double)X.dims[k];
  return c < 9.0e18;
}

FibreIndex fibre_index_carve(const ts_tensor& X, int mode, Bump& b) {
  FibreIndex F{};
  F.order = X.order;
  F.mode = mode;
  int64_t st = 1;
  for (int k = X.order - 1; k >= 0; --k) {
    F.stride[k] = k == mode ? 0 : st;
    if (k != mode) st *= X.dims[k];
  }
  const int64_t cap = fibre_index_capacity(X.nnz);
  F.mask = (uint64_t)cap - 1;
  F.keys = b.take<unsigned long long>((size_t)cap);
  F.beg = b.take<int32_t>((size_t)cap + 1);
  F.cur = b.take<int32_t>((size_t)cap);
  F.pos = b.take<int32_t>((size_t)(X.nnz > 0 ? X.nnz : 1));
  F.val = b.take<char>((size_t)(X.nnz > 0 ? X.nnz : 1) * dtype_size(X.dtype));
  F.part = b.take<int32_t>((size_t)(cap / kScanChunk) + 2);
  return F;
}

ts_status launch_fibre_index_build(const ts_tensor& X, const FibreIndex& F, int* flag,
                                   cudaStream_t st) {
  const int64_t cap = (int64_t)F.mask + 1;
  TS_CUDA(cudaMemsetAsync(F.keys, 0xFF, (size_t)cap * sizeof(unsigned long long), st));
  TS_CUDA(cudaMemsetAsync(F.cur, 0, (size_t)cap * sizeof(int32_t), st));
  const int64_t nnz = X.nnz;
  const int grid = (int)std::min<int64_t>(std::max<int64_t>(ceil_div(nnz, 256), 1), 152 * 16);
  if (nnz > 0) {
    k_fib_insert<<<grid, 256, 0, st>>>(X.indices, nnz, F, nullptr, flag);
    TS_LAUNCH_CHECK();
  }
  const int64_t nb = cap / kScanChunk + (cap % kScanChunk ? 1 : 0);
  k_scan_partials<<<(unsigned)nb, kScanThreads, 0, st>>>(F.cur, cap, F.part);
  TS_LAUNCH_CHECK();
  k_scan_top<<<1, 1024, 0, st>>>(F.part, nb);
  TS_LAUNCH_CHECK();
  k_scan_apply<<<(unsigned)nb, kScanThreads, 0, st>>>(F.cur, cap, F.part, nb, F.beg);
  TS_LAUNCH_CHECK();
  TS_CUDA(cudaMemsetAsync(F.cur, 0, (size_t)cap * sizeof(int32_t), st));
  if (nnz > 0) {
    if (X.dtype == TS_F64)
      k_fib_fill<double><<<grid, 256, 0, st>>>(X.indices, static_cast<const double*>(X.values),
                                               nnz, F, flag);
    else
      k_fib_fill<float><<<grid, 256, 0, st>>>(X.indices, static_cast<const float*>(X.values), nnz,
                                              F, flag);
    TS_LAUNCH_CHECK();
  }
  return TS_OK;
}

ts_status launch_fibre_keys(const ts_tensor& X, const FibreIndex& F, int32_t* eslot, int* flag,
                            cudaStream_t st) {
  const int64_t cap = (int64_t)F.mask + 1;
  TS_CUDA(cudaMemsetAsync(F.keys, 0xFF, (size_t)cap * sizeof(unsigned long long), st));
  const int64_t nnz = X.nnz;
  const int grid = (int)std::min<int64_t>(std::max<int64_t>(ceil_div(nnz, 256), 1), 152 * 16);
  if (nnz > 0) {
    k_fib_insert<<<grid, 256, 0, st>>>(X.indices, nnz, F, eslot, flag);
    TS_LAUNCH_CHECK();
  }
  return TS_OK;
}

}  // namespace ts
