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

// Row j: weight, Z row (Kronecker product of sampled factor rows), Y row (fibre).
template <typename T>
__global__ void k_lev_gather(LevDesc d, int m, int ncols, const T* __restrict__ X,
                             const int32_t* __restrict__ samples, const double* __restrict__ prob,
                             T* __restrict__ Z, T* __restrict__ Y) {
  const int j = blockIdx.x;
  const int nm1 = d.order - 1;
  __shared__ double w;
  __shared__ long base;
  if (threadIdx.x == 0) {
    double p = 1.0;
    for (int jj = 0; jj < nm1; ++jj) p = p * prob[(long)jj * m + j];
    w = 1.0 / sqrt((double)m * p);
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
  long sn = 1;
  for (int k = d.mode + 1; k < d.order; ++k) sn *= d.dims[k];
  for (int t = threadIdx.x; t < d.dims[d.mode]; t += blockDim.x)
    Y[(long)j * d.dims[d.mode] + t] = (T)((double)X[base + (long)t * sn] * w);
}

size_t leverage_scratch_doubles(const ts_tensor& X, int mode, int m) {
  size_t s = 0;
  for (int k = 0; k < X.order; ++k)
    if (k != mode) s += (size_t)X.dims[k];
  return 2 * s + (size_t)(X.order - 1) * m;
}

template <typename T>
ts_status launch_leverage(const ts_tensor& X, int mode, const int* ranks, const T* const* factors,
                          int m, uint64_t seed, int sweep, T* Z, T* Y, int32_t* samples,
                          double* scratch, cudaStream_t st) {
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
  k_lev_sample<T><<<X.order - 1, 256, 0, st>>>(d, m, seed, sweep, ell, cdf, samples, prob);
  TS_LAUNCH_CHECK();
  k_lev_gather<T><<<m, 128, 0, st>>>(d, m, ncols, static_cast<const T*>(X.values), samples, prob,
                                     Z, Y);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

template ts_status launch_leverage<float>(const ts_tensor&, int, const int*, const float* const*,
                                          int, uint64_t, int, float*, float*, int32_t*, double*,
                                          cudaStream_t);
template ts_status launch_leverage<double>(const ts_tensor&, int, const int*,
                                           const double* const*, int, uint64_t, int, double*,
                                           double*, int32_t*, double*, cudaStream_t);

}  // namespace ts
