// Leverage-score sampling for a Kronecker-structured left-hand side (Sec. 3.2).
// The score of row (i_k)_{k != n} of P^(n) is the product of the factor scores
// (Kronecker leverage lemma), so every i_k is drawn independently from
// p^(k) = l(A^(k)) / sum l(A^(k)); row j of the sketch is rescaled by
// 1 / sqrt(m p_j) (importance-sampling definition).
#include "internal.cuh"

namespace ts {

struct LevDesc {
  int order;
  int mode;
  int64_t dims[TS_MAX_ORDER];
  int ranks[TS_MAX_ORDER];
  const void* factors[TS_MAX_ORDER];
  int64_t off[TS_MAX_ORDER];  // offset of mode k's scores in the scratch
};

// Block j handles the j-th mode k != n: scores, running CDF (index order, FP64,
// one thread so the summation order is the plain left-to-right one), and the m
// inverse-CDF draws.
template <typename T>
__global__ void k_lev_sample(LevDesc d, int m, uint64_t seed, int sweep, double* ell, double* cdf,
                             int32_t* samples, double* prob) {
  int k = -1, jj = -1;
  for (int t = 0, c = 0; t < d.order; ++t) {
    if (t == d.mode) continue;
    if (c == (int)blockIdx.x) { k = t; jj = c; }
    ++c;
  }
  const int s = (int)d.dims[k];
  const int R = d.ranks[k];
  const T* A = static_cast<const T*>(d.factors[k]);
  double* el = ell + d.off[k];
  double* cd = cdf + d.off[k];
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    double acc = 0;
    for (int r = 0; r < R; ++r) {
      const double a = (double)A[(long)i * R + r];
      acc = __dadd_rn(acc, __dmul_rn(a, a));  // no FMA: the oracle rounds the square first
    }
    el[i] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double run = 0;
    for (int i = 0; i < s; ++i) {
      run = run + el[i];
      cd[i] = run;
    }
  }
  __syncthreads();
  const double total = cd[s - 1];
  const uint64_t key = object_key(seed, make_tag(TS_PURPOSE_LEV_UNIFORM, sweep, d.mode, k));
  const int nm1 = d.order - 1;
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    const double target = uniform01(key, (uint64_t)j) * total;
    int lo = 0, hi = s - 1;  // smallest i with cdf_i > target
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (cd[mid] > target) hi = mid; else lo = mid + 1;
    }
    samples[(long)j * nm1 + jj] = lo;
    prob[(long)jj * m + j] = el[lo] / total;
  }
}

// ---------------------------------------------------------------- deterministic selection

// Block-wide exclusive prefix sum of one value per thread (blockDim.x <= 1024); returns
// this thread's prefix and writes the total to *total.
__device__ __forceinline__ long block_exclusive_scan(long v, long* warp_sums, long* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    long t = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) warp_sums[lane] = t;  // inclusive warp totals
  }
  __syncthreads();
  const long base = warp ? warp_sums[warp - 1] : 0;
  *total = warp_sums[nw - 1];
  __syncthreads();
  return base + x - v;
}

// The "Lev-fix" variant of Sec. 3.2: the m multi-indices (i_k)_{k != n} of largest
// score prod_k l_k(i_k) (modes ascending, FP64 products rounded left to right), ties to
// the lower C-order linear index, written to samples in ascending linear index.  One
// block.  The m-th largest score is found by a radix select on the bit patterns of the
// (non-negative) scores, 8 bits at a time from the top; each thread then owns a
// contiguous chunk of candidates and two prefix sums place the selected ones in order.
// Rows j >= min(m, C) get the multi-index 0 and are zeroed by the gather.
__global__ void __launch_bounds__(1024) k_lev_select_det(LevDesc d, int m, long C,
                                                          const double* __restrict__ ell,
                                                          double* __restrict__ score,
                                                          int32_t* __restrict__ samples) {
  __shared__ unsigned hist[256];
  __shared__ long warp_sums[32];
  __shared__ unsigned long long s_prefix;
  __shared__ long s_above;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int nm1 = d.order - 1;
  int km[TS_MAX_ORDER], sz[TS_MAX_ORDER];
  for (int k = 0, j = 0; k < d.order; ++k)
    if (k != d.mode) {
      km[j] = k;
      sz[j] = (int)d.dims[k];
      ++j;
    }
  // scores of every candidate (C order over the modes k != n, last fastest)
  for (long c = tid; c < C; c += nthr) {
    long rem = c;
    int idx[TS_MAX_ORDER];
    for (int j = nm1 - 1; j >= 0; --j) {
      idx[j] = (int)(rem % sz[j]);
      rem /= sz[j];
    }
    double p = 1.0;
    for (int j = 0; j < nm1; ++j) p = __dmul_rn(p, ell[d.off[km[j]] + idx[j]]);
    score[c] = p;
  }
  const long want = m < C ? m : C;
  if (tid == 0) {
    s_prefix = 0;
    s_above = 0;
  }
  __syncthreads();
  // radix select: after the loop s_prefix holds the bits of the want-th largest score
  for (int shift = 56; shift >= 0; shift -= 8) {
    for (int i = tid; i < 256; i += nthr) hist[i] = 0;
    __syncthreads();
    const unsigned long long pre = s_prefix;
    const unsigned long long mask = shift == 56 ? 0ull : (~0ull << (shift + 8));
    for (long c = tid; c < C; c += nthr) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(score[c]);
      if ((b & mask) == pre) atomicAdd(&hist[(b >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (tid == 0) {
      long above = s_above;
      int digit = 255;
      for (; digit > 0; --digit) {
        if (above + (long)hist[digit] >= want) break;
        above += hist[digit];
      }
      s_above = above;  // candidates strictly above the chosen digit so far
      s_prefix = pre | ((unsigned long long)digit << shift);
    }
    __syncthreads();
  }
  const unsigned long long kth = s_prefix;
  const long need_ties = want - s_above;  // the lowest-index candidates equal to kth
  // chunk per thread, in index order
  const long per = (C + nthr - 1) / nthr;
  const long c0 = (long)tid * per, c1 = c0 + per < C ? c0 + per : C;
  long ties = 0;
  for (long c = c0; c < c1; ++c)
    ties += (unsigned long long)__double_as_longlong(score[c]) == kth;
  long tot;
  long tie_base = block_exclusive_scan(ties, warp_sums, &tot);
  long sel = 0, tr = tie_base;
  for (long c = c0; c < c1; ++c) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(score[c]);
    if (b > kth) ++sel;
    else if (b == kth) sel += (tr++ < need_ties);
  }
  long out = block_exclusive_scan(sel, warp_sums, &tot);
  tr = tie_base;
  for (long c = c0; c < c1; ++c) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(score[c]);
    bool take = b > kth;
    if (b == kth) take = tr++ < need_ties;
    if (!take) continue;
    long rem = c;
    for (int j = nm1 - 1; j >= 0; --j) {
      samples[out * nm1 + j] = (int32_t)(rem % sz[j]);
      rem /= sz[j];
    }
    ++out;
  }
  for (long j = want + tid; j < m; j += nthr)
    for (int q = 0; q < nm1; ++q) samples[j * nm1 + q] = 0;
}

// Row j: weight, Z row (Kronecker product of sampled factor rows), Y row (fibre).
// unit: weights 1 for rows j < nrows and 0 beyond (deterministic selection).
template <typename T>
__global__ void k_lev_gather(LevDesc d, int m, int ncols, const T* __restrict__ X,
                             const int32_t* __restrict__ samples, const double* __restrict__ prob,
                             T* __restrict__ Z, T* __restrict__ Y, int unit, long nrows,
                             FibreIndex F, int coo) {
  const int j = blockIdx.x;
  const int nm1 = d.order - 1;
  __shared__ double w;
  __shared__ long base;
  if (threadIdx.x == 0) {
    double p = 1.0;
    if (!unit)
      for (int jj = 0; jj < nm1; ++jj) p = p * prob[(long)jj * m + j];
    w = unit ? (j < nrows ? 1.0 : 0.0) : 1.0 / sqrt((double)m * p);
    long b = 0, stride = 1;
    for (int k = d.order - 1, jj = nm1 - 1; k >= 0; --k) {
      if (k != d.mode) {
        b += (long)samples[(long)j * nm1 + jj] * stride;
        --jj;
      }
      stride *= d.dims[k];
    }
    base = b;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
    double v = 1.0;
    int x = c;
    for (int k = d.order - 1, jj = nm1 - 1; k >= 0; --k) {
      if (k == d.mode) continue;
      const int rk = x % d.ranks[k];
      x /= d.ranks[k];
      const T* A = static_cast<const T*>(d.factors[k]);
      v *= (double)A[(long)samples[(long)j * nm1 + jj] * d.ranks[k] + rk];
      --jj;
    }
    Z[(long)c * m + j] = (T)(v * w);
  }
  if (coo) {
    // the sampled fibre's nonzeros from the index; Y was zeroed, repeated coordinates add
    __shared__ int32_t fb[2];
    if (threadIdx.x == 0) {
      unsigned long long key = 0;
      for (int k = 0, jj = 0; k < d.order; ++k)
        if (k != d.mode) key += (unsigned long long)samples[(long)j * nm1 + jj++] * F.stride[k];
      uint64_t h = mix64(key) & F.mask;
      fb[0] = fb[1] = 0;
      for (uint64_t p = 0; p <= F.mask; ++p) {
        const unsigned long long cur = F.keys[h];
        if (cur == key) {
          fb[0] = F.beg[h];
          fb[1] = F.beg[h + 1];
          break;
        }
        if (cur == ~0ull) break;  // empty fibre
        h = (h + 1) & F.mask;
      }
    }
    __syncthreads();
    if (w != 0.0) {
      const T* val = static_cast<const T*>(F.val);
      T* yr = Y + (long)j * d.dims[d.mode];
      const unsigned sn = (unsigned)d.dims[d.mode];
      for (int p = fb[0] + threadIdx.x; p < fb[1]; p += blockDim.x) {
        const unsigned i = (unsigned)F.pos[p];
        if (i < sn) atomicAdd(yr + i, (T)((double)val[p] * w));  // coordinates out of range drop
      }
    }
    return;
  }
  long sn = 1;
  for (int k = d.mode + 1; k < d.order; ++k) sn *= d.dims[k];
  for (int t = threadIdx.x; t < d.dims[d.mode]; t += blockDim.x)
    Y[(long)j * d.dims[d.mode] + t] = (T)((double)X[base + (long)t * sn] * w);
}

int64_t leverage_det_candidates(const ts_tensor& X, int mode) {
  double c = 1;
  for (int k = 0; k < X.order; ++k)
    if (k != mode) c *= (double)X.dims[k];
  return c > (double)kLevDetMaxCandidates ? -1 : (int64_t)c;
}

size_t leverage_scratch_doubles(const ts_tensor& X, int mode, int m) {
  size_t s = 0;
  for (int k = 0; k < X.order; ++k)
    if (k != mode) s += (size_t)X.dims[k];
  // + C: the deterministic selection's score of every multi-index (when it can run)
  const int64_t C = leverage_det_candidates(X, mode);
  return 2 * s + (size_t)(X.order - 1) * m + (C > 0 ? (size_t)C : 0);
}

template <typename T>
ts_status launch_leverage(const ts_tensor& X, int mode, const int* ranks, const T* const* factors,
                          int m, uint64_t seed, int sweep, T* Z, T* Y, int32_t* samples,
                          double* scratch, cudaStream_t st, bool det, const FibreIndex* fib) {
  LevDesc d{};
  d.order = X.order;
  d.mode = mode;
  size_t off = 0;
  int ncols = 1;
  for (int k = 0; k < X.order; ++k) {
    d.dims[k] = X.dims[k];
    d.ranks[k] = ranks[k];
    d.factors[k] = factors[k];
    if (k != mode) {
      d.off[k] = (int64_t)off;
      off += (size_t)X.dims[k];
      ncols *= ranks[k];
    }
  }
  double* ell = scratch;
  double* cdf = scratch + off;
  double* prob = scratch + 2 * off;
  long C = 1;
  if (det) {
    C = (long)leverage_det_candidates(X, mode);
    if (C < 0)
      return fail(TS_ERR_UNSUPPORTED,
                  "deterministic leverage: more than %lld candidate rows for mode %d",
                  (long long)kLevDetMaxCandidates, mode);
  }
  // deterministic: the scores only (no draws), then the selection
  k_lev_sample<T><<<X.order - 1, 256, 0, st>>>(d, det ? 0 : m, seed, sweep, ell, cdf, samples,
                                                prob);
  TS_LAUNCH_CHECK();
  if (det) {
    k_lev_select_det<<<1, 1024, 0, st>>>(d, m, C, ell, prob + (size_t)(X.order - 1) * m,
                                          samples);
    TS_LAUNCH_CHECK();
  }
  const bool coo = X.format == TS_COO;
  if (coo && !fib) return fail(TS_ERR_INVALID_ARG, "leverage sketch of a COO tensor: no index");
  FibreIndex F{};
  if (coo) {
    F = *fib;
    TS_CUDA(cudaMemsetAsync(Y, 0, (size_t)m * X.dims[mode] * sizeof(T), st));
  }
  // COO: 512 threads per sampled fibre (the heavy fibres of skewed data hold 10^4+ nonzeros)
  k_lev_gather<T><<<m, coo ? 512 : 128, 0, st>>>(
      d, m, ncols, coo ? nullptr : static_cast<const T*>(X.values), samples, prob, Z, Y,
      det ? 1 : 0, det ? (m < C ? (long)m : C) : (long)m, F, coo ? 1 : 0);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

template ts_status launch_leverage<float>(const ts_tensor&, int, const int*, const float* const*,
                                          int, uint64_t, int, float*, float*, int32_t*, double*,
                                          cudaStream_t, bool, const FibreIndex*);
template ts_status launch_leverage<double>(const ts_tensor&, int, const int*,
                                           const double* const*, int, uint64_t, int, double*,
                                           double*, int32_t*, double*, cudaStream_t, bool,
                                           const FibreIndex*);

}  // namespace ts
