// Relative residual ||T - T~||_F / ||T||_F of a Tucker model against a COO tensor
// (Sec. 7 fitness f = 1 - residual), without forming T~:
//   ||T - T~||^2 = ||T||^2 - 2 <T, T~> + ||T~||^2
//   ||T||^2  over distinct coordinates, repeated ones added first (once per tensor):
//            every nonzero finds the hash slot of its mode-nf fibre (the fibre index's
//            keys), and (fibre slot, i_nf) keys a second hash table that sums the repeats
//   <T, T~>  = sum over stored entries of v_e T~(i_e) (linear in the entries, so
//            repeats need no merging); T~(i) = sum_r C(r) prod_n A^(n)(i_n, r_n) with
//            the core in shared memory and the last mode's factor row in registers
//   ||T~||^2 = <C, C x_1 G_1 ... x_N G_N>, G_n = A^(n)T A^(n) (exact without
//            orthonormal factors)
// Every sum across threads is FP64; the per-entry value T~(i) is formed in the data type.
#include "internal.cuh"

namespace ts {

namespace {

constexpr unsigned long long kEmptyKey = ~0ull;

__device__ __forceinline__ double block_sum_d(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
  return t;  // valid in thread 0
}

struct CooExtent {
  int order;
  int64_t dims[TS_MAX_ORDER];
};

// Adds every nonzero's value into the slot of key (fibre slot, i_nf) of the value table.
// Entries with a coordinate outside [0, dims[k]) are skipped, as in <T, T~> and the input
// sketch (their fibre key could alias another fibre's).
template <typename T>
__global__ void k_merge_repeats(const int32_t* __restrict__ idx, const T* __restrict__ vals,
                                int64_t nnz, int nf, CooExtent ext,
                                const int32_t* __restrict__ eslot,
                                unsigned long long* __restrict__ vkeys, double* __restrict__ vsum,
                                uint64_t vmask, int* flag) {
  const int64_t sn = ext.dims[nf];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    bool ok = true;
    for (int k = 0; k < ext.order; ++k) {
      const int32_t i = idx[(int64_t)k * nnz + e];
      ok &= (i >= 0) & (i < ext.dims[k]);
    }
    if (!ok) continue;
    const unsigned long long key = (unsigned long long)(unsigned)eslot[e] * (unsigned long long)sn +
                                   (unsigned long long)(unsigned)idx[(int64_t)nf * nnz + e];
    uint64_t g = mix64(key) & vmask;
    bool placed = false;
    for (uint64_t q = 0; q <= vmask; ++q) {
      unsigned long long cur = __ldcg(vkeys + g);
      if (cur == kEmptyKey) cur = atomicCAS(vkeys + g, kEmptyKey, key);
      if (cur == kEmptyKey || cur == key) {
        atomicAdd(vsum + g, (double)vals[e]);
        placed = true;
        break;
      }
      g = (g + 1) & vmask;
    }
    if (!placed && flag) atomicExch(flag, 2);
  }
}

__global__ void k_sum_squares(const double* __restrict__ v, int64_t n, double* out) {
  __shared__ double sh[32];
  double s = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += v[i] * v[i];
  s = block_sum_d(s, sh);
  if (threadIdx.x == 0) atomicAdd(out, s);
}

struct CooModel {
  int order;
  int64_t dims[TS_MAX_ORDER];
  int ranks[TS_MAX_ORDER];
  const void* factors[TS_MAX_ORDER];
  int npre;  // prod_{k < order-1} ranks[k]
};

// Entries with a coordinate outside [0, dims[k]) are skipped (as in the input sketch).
__device__ __forceinline__ bool entry_in_range(const int32_t* __restrict__ idx, int64_t nnz,
                                               int64_t e, const CooModel& d) {
  bool ok = true;
  for (int k = 0; k < d.order; ++k) {
    const int32_t i = idx[(int64_t)k * nnz + e];
    ok &= (i >= 0) & (i < d.dims[k]);
  }
  return ok;
}

// <T, T~>: one thread per stored entry.  RL >= ranks[last] (the last factor row in
// registers, zero-padded; the core rows in shared memory are padded to match).
template <typename T, int RL>
__global__ void __launch_bounds__(256) k_coo_inner(const int32_t* __restrict__ idx,
                                                   const T* __restrict__ vals, int64_t nnz,
                                                   CooModel d, const T* __restrict__ core,
                                                   double* out) {
  extern __shared__ unsigned char smraw[];
  T* sc = reinterpret_cast<T*>(smraw);
  __shared__ double sh[32];
  const int N = d.order, L = N - 1, RLr = d.ranks[L];
  const int ctot = d.npre * RLr;
  for (int i = threadIdx.x; i < ctot + RL; i += blockDim.x) sc[i] = i < ctot ? core[i] : (T)0;
  __syncthreads();
  const T* AL = static_cast<const T*>(d.factors[L]);
  double acc = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (!entry_in_range(idx, nnz, e, d)) continue;
    T al[RL];
    const int64_t il = idx[(int64_t)L * nnz + e];
#pragma unroll
    for (int r = 0; r < RL; ++r) al[r] = r < RLr ? AL[il * RLr + r] : (T)0;
    int64_t ik[TS_MAX_ORDER];
    int rk[TS_MAX_ORDER];
    T pp[TS_MAX_ORDER];  // pp[k] = prod_{j <= k} A^(j)(i_j, r_j)
    for (int k = 0; k < L; ++k) {
      ik[k] = idx[(int64_t)k * nnz + e];
      rk[k] = 0;
      const T a = static_cast<const T*>(d.factors[k])[ik[k] * d.ranks[k]];
      pp[k] = k ? pp[k - 1] * a : a;
    }
    T s = 0;
    for (int c = 0; c < d.npre; ++c) {
      const T* crow = sc + (long)c * RLr;
      T inner = 0;
#pragma unroll
      for (int r = 0; r < RL; ++r) inner += crow[r] * al[r];
      s += pp[L - 1] * inner;
      int k = L - 1;  // odometer over (r_0, ..., r_{L-1}), last fastest
      while (k >= 0 && ++rk[k] == d.ranks[k]) rk[k--] = 0;
      if (k < 0) break;
      for (int j = k; j < L; ++j) {
        const T a = static_cast<const T*>(d.factors[j])[ik[j] * d.ranks[j] + rk[j]];
        pp[j] = j ? pp[j - 1] * a : a;
      }
    }
    acc += (double)s * (double)vals[e];
  }
  acc = block_sum_d(acc, sh);
  if (threadIdx.x == 0) atomicAdd(out, acc);
}

// Unrolled form for order N <= 4 with every rank <= RR: the core zero-padded to RR^N in
// shared memory; the rows of the last two modes in registers and their RR^2 terms fully
// unrolled (the last mode innermost); the leading modes looped, their factor entries
// read through L1.
template <typename T, int N, int RR>
__global__ void __launch_bounds__(256) k_coo_inner_fixed(const int32_t* __restrict__ idx,
                                                         const T* __restrict__ vals, int64_t nnz,
                                                         CooModel d, const T* __restrict__ core,
                                                         double* out) {
  static_assert(N >= 2 && N <= 4, "orders 2..4");
  constexpr int P = N == 2 ? RR * RR : N == 3 ? RR * RR * RR : RR * RR * RR * RR;
  extern __shared__ unsigned char smraw[];
  T* sc = reinterpret_cast<T*>(smraw);
  __shared__ double sh[32];
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    int rem = i;
    long src = 0, stride = 1;
    bool in = true;
    for (int k = N - 1; k >= 0; --k) {
      const int rk = rem % RR;
      rem /= RR;
      in &= rk < d.ranks[k];
      src += rk * stride;
      stride *= d.ranks[k];
    }
    sc[i] = in ? core[src] : (T)0;
  }
  __syncthreads();
  double acc = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (!entry_in_range(idx, nnz, e, d)) continue;
    T a[2][RR];  // rows of modes N-2 and N-1
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int k = N - 2 + q;
      const T* A = static_cast<const T*>(d.factors[k]);
      const int64_t i = idx[(int64_t)k * nnz + e];
      const int R = d.ranks[k];
#pragma unroll
      for (int r = 0; r < RR; ++r) a[q][r] = r < R ? __ldg(A + i * R + r) : (T)0;
    }
    // one RR x RR block of the core per prefix (r_0, ..., r_{N-3}) of the leading modes,
    // weighted by the product of their factor entries
    auto block_sum = [&](const T* blk) -> T {
      T s2 = 0;
#pragma unroll
      for (int r2 = 0; r2 < RR; ++r2) {
        T inner = 0;
#pragma unroll
        for (int r3 = 0; r3 < RR; ++r3) inner += blk[r2 * RR + r3] * a[1][r3];
        s2 += a[0][r2] * inner;
      }
      return s2;
    };
    T s = 0;
    if constexpr (N == 2) {
      s = block_sum(sc);
    } else {
      const T* A0 = static_cast<const T*>(d.factors[0]);
      const int R0 = d.ranks[0];
      const int64_t i0 = idx[e];
      if constexpr (N == 3) {
        for (int r0 = 0; r0 < R0; ++r0)
          s += __ldg(A0 + i0 * R0 + r0) * block_sum(sc + r0 * RR * RR);
      } else {
        // mode 1's row in registers too: the RR blocks of one r0 unrolled
        T a1[RR];
        const T* A1 = static_cast<const T*>(d.factors[1]);
        const int R1 = d.ranks[1];
        const int64_t i1 = idx[nnz + e];
#pragma unroll
        for (int r = 0; r < RR; ++r) a1[r] = r < R1 ? __ldg(A1 + i1 * R1 + r) : (T)0;
        for (int r0 = 0; r0 < R0; ++r0) {
          T s1 = 0;
#pragma unroll
          for (int r1 = 0; r1 < RR; ++r1) s1 += a1[r1] * block_sum(sc + (r0 * RR + r1) * RR * RR);
          s += __ldg(A0 + i0 * R0 + r0) * s1;
        }
      }
    }
    acc += (double)s * (double)vals[e];
  }
  acc = block_sum_d(acc, sh);
  if (threadIdx.x == 0) atomicAdd(out, acc);
}

// G_n = A^(n)T A^(n): block (a, b, n) sums A(:, a) A(:, b) over the rows in FP64.
template <typename T>
__global__ void k_gram_cols(CooModel d, T* G, int gstride) {
  __shared__ double sh[32];
  const int n = blockIdx.z;
  const int R = d.ranks[n];
  const int a = blockIdx.x, b = blockIdx.y;
  if (a >= R || b >= R) return;
  const T* A = static_cast<const T*>(d.factors[n]);
  double s = 0;
  for (int64_t i = threadIdx.x; i < d.dims[n]; i += blockDim.x)
    s += (double)A[i * R + a] * (double)A[i * R + b];
  s = block_sum_d(s, sh);
  if (threadIdx.x == 0) G[(long)n * gstride + a * R + b] = (T)s;
}

// out = in x_k G (G square R x R): in, out are (pre x R x post), C order.
template <typename T>
__global__ void k_ttm_square(long pre, int R, long post, const T* __restrict__ in,
                             const T* __restrict__ G, T* __restrict__ out) {
  const long total = pre * R * post;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long y = e % post;
    const long xi = e / post;
    const int i = (int)(xi % R);
    const long x = xi / R;
    const T* src = in + x * R * post + y;
    double acc = 0;
    for (int r = 0; r < R; ++r) acc += (double)G[i * R + r] * (double)src[r * post];
    out[e] = (T)acc;
  }
}

// acc[2] = <C, M> = ||T~||^2; the residual from *t2 = ||T||^2 and acc[1] = <T, T~>.
template <typename T>
__global__ void k_fit_coo_final(const T* __restrict__ C, const T* __restrict__ M, long n,
                                const double* __restrict__ t2, double* acc, double* residual) {
  __shared__ double sh[32];
  double s = 0;
  for (long i = threadIdx.x; i < n; i += blockDim.x) s += (double)C[i] * (double)M[i];
  s = block_sum_d(s, sh);
  if (threadIdx.x == 0) {
    const double tt = *t2;
    const double r2 = tt - 2.0 * acc[1] + s;
    acc[2] = s;
    *residual = tt > 0 ? sqrt((r2 > 0 ? r2 : 0.0) / tt) : 0.0;  // as the dense form: 0 for T = 0
  }
}

int fit_coo_mode(const ts_tensor& X) {
  int nf = 0;
  for (int k = 1; k < X.order; ++k)
    if (X.dims[k] > X.dims[nf]) nf = k;
  return nf;
}

}  // namespace

bool fit_coo_supported(const ts_tensor& X) {
  if (X.order < 2 || X.nnz >= (int64_t(1) << 30)) return false;
  return fibre_keys_fit(X, fit_coo_mode(X));
}

bool fit_coo_model_ok(const ts_tensor& X, const int* ranks) {
  long ctot = 1;
  for (int k = 0; k < X.order; ++k) ctot *= ranks[k];
  return ranks[X.order - 1] <= 64 && (ctot + 64) * (long)dtype_size(X.dtype) <= 200 * 1024;
}

FitCooWork fit_coo_carve(const ts_tensor& X, const int* ranks, Bump& b) {
  FitCooWork w{};
  const int nf = fit_coo_mode(X);
  const int64_t cap = fibre_index_capacity(X.nnz);
  w.F.order = X.order;
  w.F.mode = nf;
  int64_t st = 1;
  for (int k = X.order - 1; k >= 0; --k) {
    w.F.stride[k] = k == nf ? 0 : st;
    if (k != nf) st *= X.dims[k];
  }
  w.F.mask = (uint64_t)cap - 1;
  w.F.keys = b.take<unsigned long long>((size_t)cap);
  w.eslot = b.take<int32_t>((size_t)(X.nnz > 0 ? X.nnz : 1));
  w.vmask = (uint64_t)cap - 1;
  w.vkeys = b.take<unsigned long long>((size_t)cap);
  w.vsum = b.take<double>((size_t)cap);
  long ctot = 1;
  int gmax = 0;
  for (int k = 0; k < X.order; ++k) {
    ctot *= ranks[k];
    if (ranks[k] * ranks[k] > gmax) gmax = ranks[k] * ranks[k];
  }
  const size_t ts = dtype_size(X.dtype);
  w.gstride = gmax;
  w.G = b.take<char>((size_t)X.order * gmax * ts);
  w.M1 = b.take<char>((size_t)ctot * ts);
  w.M2 = b.take<char>((size_t)ctot * ts);
  w.acc = b.take<double>(4);
  return w;
}

ts_status launch_fit_coo_norm(const ts_tensor& X, const FitCooWork& w, int* flag,
                              cudaStream_t st) {
  TS_TRY(launch_fibre_keys(X, w.F, w.eslot, flag, st));
  const int64_t cap = (int64_t)w.vmask + 1;
  TS_CUDA(cudaMemsetAsync(w.vkeys, 0xFF, (size_t)cap * sizeof(unsigned long long), st));
  TS_CUDA(cudaMemsetAsync(w.vsum, 0, (size_t)cap * sizeof(double), st));
  TS_CUDA(cudaMemsetAsync(w.acc, 0, 4 * sizeof(double), st));
  const int grid = (int)std::min<int64_t>(std::max<int64_t>(ceil_div(X.nnz, 256), 1), 152 * 16);
  CooExtent ext{};
  ext.order = X.order;
  for (int k = 0; k < X.order; ++k) ext.dims[k] = X.dims[k];
  if (X.nnz > 0) {
    if (X.dtype == TS_F64)
      k_merge_repeats<double><<<grid, 256, 0, st>>>(X.indices,
                                                    static_cast<const double*>(X.values), X.nnz,
                                                    w.F.mode, ext, w.eslot, w.vkeys, w.vsum,
                                                    w.vmask, flag);
    else
      k_merge_repeats<float><<<grid, 256, 0, st>>>(X.indices, static_cast<const float*>(X.values),
                                                   X.nnz, w.F.mode, ext, w.eslot, w.vkeys, w.vsum,
                                                   w.vmask, flag);
    TS_LAUNCH_CHECK();
  }
  k_sum_squares<<<(int)std::min<int64_t>(ceil_div(cap, 256), 152 * 8), 256, 0, st>>>(w.vsum, cap,
                                                                                     w.acc + 3);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

template <typename T, int RL>
static ts_status inner_launch(const ts_tensor& X, const CooModel& d, const T* core, double* out,
                              cudaStream_t st) {
  const size_t smem = ((size_t)d.npre * d.ranks[X.order - 1] + RL) * sizeof(T);
  if (smem > 200 * 1024)
    return fail(TS_ERR_UNSUPPORTED, "COO fitness: core of %zu bytes exceeds shared memory", smem);
  if (smem > 48 * 1024)
    TS_CUDA(cudaFuncSetAttribute(k_coo_inner<T, RL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  const int grid = (int)std::min<int64_t>(std::max<int64_t>(ceil_div(X.nnz, 256), 1), 152 * 8);
  k_coo_inner<T, RL><<<grid, 256, smem, st>>>(X.indices, static_cast<const T*>(X.values), X.nnz,
                                              d, core, out);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

template <typename T>
ts_status launch_fit_coo(const ts_tensor& X, const int* ranks, const T* core,
                         const T* const* factors, const FitCooWork& w, double* residual,
                         cudaStream_t st) {
  const int N = X.order;
  CooModel d{};
  d.order = N;
  d.npre = 1;
  for (int k = 0; k < N; ++k) {
    d.dims[k] = X.dims[k];
    d.ranks[k] = ranks[k];
    d.factors[k] = factors[k];
    if (k < N - 1) d.npre *= ranks[k];
  }
  TS_CUDA(cudaMemsetAsync(w.acc + 1, 0, sizeof(double), st));
  const int RLr = ranks[N - 1];
  int rmax = 0;
  for (int k = 0; k < N; ++k) rmax = std::max(rmax, ranks[k]);
  const int grid = (int)std::min<int64_t>(std::max<int64_t>(ceil_div(X.nnz, 256), 1), 152 * 8);
  const T* vals = static_cast<const T*>(X.values);
  auto fixed = [&](auto kern, int P) -> ts_status {
    const size_t smem = (size_t)P * sizeof(T);
    if (smem > 48 * 1024)
      TS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, 256, smem, st>>>(X.indices, vals, X.nnz, d, core, w.acc + 1);
    TS_LAUNCH_CHECK();
    return TS_OK;
  };
  if (N == 4 && rmax <= 8) TS_TRY(fixed(k_coo_inner_fixed<T, 4, 8>, 4096));
  else if (N == 3 && rmax <= 8) TS_TRY(fixed(k_coo_inner_fixed<T, 3, 8>, 512));
  else if (N == 3 && rmax <= 16) TS_TRY(fixed(k_coo_inner_fixed<T, 3, 16>, 4096));
  else if (N == 2 && rmax <= 16) TS_TRY(fixed(k_coo_inner_fixed<T, 2, 16>, 256));
  else if (RLr <= 8) TS_TRY((inner_launch<T, 8>(X, d, core, w.acc + 1, st)));
  else if (RLr <= 16) TS_TRY((inner_launch<T, 16>(X, d, core, w.acc + 1, st)));
  else if (RLr <= 32) TS_TRY((inner_launch<T, 32>(X, d, core, w.acc + 1, st)));
  else if (RLr <= 64) TS_TRY((inner_launch<T, 64>(X, d, core, w.acc + 1, st)));
  else return fail(TS_ERR_UNSUPPORTED, "COO fitness: last rank %d > 64", RLr);
  // ||T~||^2 = <C, C x_1 G_1 ... x_N G_N>
  int Rm = 0;
  for (int k = 0; k < N; ++k)
    if (ranks[k] > Rm) Rm = ranks[k];
  T* G = static_cast<T*>(w.G);
  k_gram_cols<T><<<dim3(Rm, Rm, N), 256, 0, st>>>(d, G, w.gstride);
  TS_LAUNCH_CHECK();
  long ctot = 1;
  for (int k = 0; k < N; ++k) ctot *= ranks[k];
  const T* in = core;
  T* bufs[2] = {static_cast<T*>(w.M1), static_cast<T*>(w.M2)};
  long pre = 1;
  for (int k = 0; k < N; ++k) {
    const long post = ctot / (pre * ranks[k]);
    T* out = bufs[k & 1];
    k_ttm_square<T><<<std::max(1, std::min(ceil_div(ctot, 256), 152 * 4)), 256, 0, st>>>(
        pre, ranks[k], post, in, G + (long)k * w.gstride, out);
    TS_LAUNCH_CHECK();
    in = out;
    pre *= ranks[k];
  }
  k_fit_coo_final<T><<<1, 256, 0, st>>>(core, in, ctot, w.acc + 3, w.acc, residual);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

template ts_status launch_fit_coo<float>(const ts_tensor&, const int*, const float*,
                                         const float* const*, const FitCooWork&, double*,
                                         cudaStream_t);
template ts_status launch_fit_coo<double>(const ts_tensor&, const int*, const double*,
                                          const double* const*, const FitCooWork&, double*,
                                          cudaStream_t);

}  // namespace ts
