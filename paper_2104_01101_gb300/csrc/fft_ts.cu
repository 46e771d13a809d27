// TensorSketch of a Kronecker chain by the FFT identity of Sec. 3.1:
//   SP = IFFT( ( (.)_j FFT(S^(j) A^(j))^T )^T ).
// Each factor column is CountSketched into shared memory (bucket/sign from the
// packed table), transformed by a shared-memory mixed-radix Stockham FFT, and the
// spectra of every column multi-index are multiplied and inverse transformed.
// Two real columns share one complex transform (x + i y), both forward and inverse.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace ts {

FftPlan make_fft_plan(int m) {
  FftPlan p{};
  p.m = m;
  p.nst = 0;
  int r = m;
  while (r % 4 == 0) { p.radix[p.nst++] = 4; r /= 4; }
  while (r % 2 == 0) { p.radix[p.nst++] = 2; r /= 2; }
  const int small[] = {3, 5, 7, 11, 13};
  for (int q : small)
    while (r % q == 0) { p.radix[p.nst++] = q; r /= q; }
  for (int q = 17; r > 1; q += 2)
    while (r % q == 0) { p.radix[p.nst++] = q; r /= q; }
  return p;
}

template <>
int fft_max_len<float>() { return 12288; }
template <>
int fft_max_len<double>() { return 6144; }

// tw[j] = exp(-2 pi i j / m), evaluated in FP64.
template <typename T>
__global__ void k_twiddles(int m, Cx<T>* __restrict__ tw) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)j / (double)m, &s, &c);
    tw[j] = Cx<T>{(T)c, (T)(-s)};
  }
}

template <typename T>
ts_status launch_twiddles(int m, Cx<T>* tw, cudaStream_t st) {
  k_twiddles<T><<<ceil_div(m, 64), 64, 0, st>>>(m, tw);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

// In-register DFT of size P (forward).  Radices 2, 3, 4 and 5 are written out (3 and 5
// pair v_r with v_{P-r}, whose twiddles are complex conjugates); the others sum the
// P x P DFT directly with twiddles tw[(r q mod P) * m/P].
template <typename T, int P>
__device__ __forceinline__ void dft_small(Cx<T> (&v)[P], const Cx<T>* __restrict__ tw, int mp) {
  if constexpr (P == 2) {
    Cx<T> a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if constexpr (P == 4) {
    Cx<T> a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    Cx<T> c = cadd(v[1], v[3]), d = csub(v[1], v[3]);
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = Cx<T>{b.x + d.y, b.y - d.x};  // b - i d
    v[3] = Cx<T>{b.x - d.y, b.y + d.x};  // b + i d
  } else if constexpr (P == 3) {
    // y0 = v0 + t, y1,2 = (v0 - t/2) -/+ i (sqrt(3)/2)(v1 - v2), t = v1 + v2
    const T h = (T)0.86602540378443865;
    const Cx<T> t = cadd(v[1], v[2]), dd = csub(v[1], v[2]);
    const Cx<T> a{v[0].x - (T)0.5 * t.x, v[0].y - (T)0.5 * t.y};
    const Cx<T> bb{h * dd.x, h * dd.y};
    v[0] = cadd(v[0], t);
    v[1] = Cx<T>{a.x + bb.y, a.y - bb.x};
    v[2] = Cx<T>{a.x - bb.y, a.y + bb.x};
  } else if constexpr (P == 5) {
    // pairs v1 +- v4, v2 +- v3 with c1,2 = cos(2 pi / 5, 4 pi / 5), s1,2 = sin(...)
    const T c1 = (T)0.30901699437494742, c2 = (T)-0.80901699437494742;
    const T s1 = (T)0.95105651629515357, s2 = (T)0.58778525229247313;
    const Cx<T> t1 = cadd(v[1], v[4]), t3 = csub(v[1], v[4]);
    const Cx<T> t2 = cadd(v[2], v[3]), t4 = csub(v[2], v[3]);
    const Cx<T> a1{v[0].x + c1 * t1.x + c2 * t2.x, v[0].y + c1 * t1.y + c2 * t2.y};
    const Cx<T> a2{v[0].x + c2 * t1.x + c1 * t2.x, v[0].y + c2 * t1.y + c1 * t2.y};
    const Cx<T> b1{s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y};
    const Cx<T> b2{s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y};
    v[0] = Cx<T>{v[0].x + t1.x + t2.x, v[0].y + t1.y + t2.y};
    v[1] = Cx<T>{a1.x + b1.y, a1.y - b1.x};  // a1 - i b1
    v[4] = Cx<T>{a1.x - b1.y, a1.y + b1.x};  // a1 + i b1
    v[2] = Cx<T>{a2.x + b2.y, a2.y - b2.x};  // a2 - i b2
    v[3] = Cx<T>{a2.x - b2.y, a2.y + b2.x};  // a2 + i b2
  } else {
    Cx<T> o[P];
#pragma unroll
    for (int q = 0; q < P; ++q) {
      Cx<T> acc = v[0];
#pragma unroll
      for (int r = 1; r < P; ++r) acc = cadd(acc, cmul(v[r], tw[((r * q) % P) * mp]));
      o[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < P; ++q) v[q] = o[q];
  }
}

// One Stockham autosort stage of radix P: butterfly j reads src[j + r m/P],
// applies exp(-2 pi i r k / (Ns P)) with k = j mod Ns, transforms, and writes
// dst[(j / Ns) Ns P + k + q Ns].
template <typename T, int P>
__device__ void fft_stage(const Cx<T>* src, Cx<T>* dst, int m, int Ns,
                          const Cx<T>* __restrict__ tw) {
  const int nb = m / P;
  const int tws = m / (Ns * P);
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    const int k = j % Ns;
    Cx<T> v[P];
#pragma unroll
    for (int r = 0; r < P; ++r) v[r] = src[j + r * nb];
    if (k > 0) {
#pragma unroll
      for (int r = 1; r < P; ++r) v[r] = cmul(v[r], tw[r * k * tws]);
    }
    dft_small<T, P>(v, tw, nb);
    const int base = (j / Ns) * Ns * P + k;
#pragma unroll
    for (int q = 0; q < P; ++q) dst[base + q * Ns] = v[q];
  }
}

// Stage of arbitrary radix P (large prime factors): one output per thread.
template <typename T>
__device__ void fft_stage_generic(const Cx<T>* src, Cx<T>* dst, int m, int Ns, int P,
                                  const Cx<T>* __restrict__ tw) {
  const int nb = m / P;
  const int tws = m / (Ns * P);
  for (int t = threadIdx.x; t < m; t += blockDim.x) {
    const int j = t / P, q = t % P;
    const int k = j % Ns;
    Cx<T> acc{0, 0};
    for (int r = 0; r < P; ++r) {
      int e = (int)(((long)r * k * tws + (long)((r * (long)q) % P) * nb) % m);
      acc = cadd(acc, cmul(src[j + r * nb], tw[e]));
    }
    dst[(j / Ns) * Ns * P + k + q * Ns] = acc;
  }
}

// Forward FFT of length plan.m held in a (b is the ping-pong buffer).  Returns
// the buffer that holds the result.  Must be called by the whole block.
template <typename T>
__device__ Cx<T>* fft_run(Cx<T>* a, Cx<T>* b, const FftPlan& plan,
                          const Cx<T>* __restrict__ tw) {
  int Ns = 1;
  const int m = plan.m;
  for (int s = 0; s < plan.nst; ++s) {
    const int P = plan.radix[s];
    switch (P) {
      case 2: fft_stage<T, 2>(a, b, m, Ns, tw); break;
      case 3: fft_stage<T, 3>(a, b, m, Ns, tw); break;
      case 4: fft_stage<T, 4>(a, b, m, Ns, tw); break;
      case 5: fft_stage<T, 5>(a, b, m, Ns, tw); break;
      case 7: fft_stage<T, 7>(a, b, m, Ns, tw); break;
      case 11: fft_stage<T, 11>(a, b, m, Ns, tw); break;
      case 13: fft_stage<T, 13>(a, b, m, Ns, tw); break;
      default: fft_stage_generic<T>(a, b, m, Ns, P, tw); break;
    }
    __syncthreads();
    Cx<T>* t = a;
    a = b;
    b = t;
    Ns *= P;
  }
  return a;
}

// Block bx: flat factor columns 2 bx (real part) and 2 bx + 1 (imaginary part).
template <typename T>
__device__ __forceinline__ void factor_spectra_body(const ChainDesc& d, const FftPlan& plan,
                                                    const Cx<T>* __restrict__ tw,
                                                    Cx<T>* __restrict__ spectra, int bx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = plan.m;
  Cx<T>* a = reinterpret_cast<Cx<T>*>(smem_raw);
  Cx<T>* b = a + m;
  const Cx<T>* twp = tw;
  if (plan.stage_tw) {  // twiddles in shared memory: every stage reads them
    Cx<T>* tws = b + m;
    for (int i = threadIdx.x; i < m; i += blockDim.x) tws[i] = tw[i];
    twp = tws;
  }
  const int c0 = 2 * bx;
  const int c1 = c0 + 1;
  for (int i = threadIdx.x; i < m; i += blockDim.x) a[i] = Cx<T>{0, 0};
  __syncthreads();
  for (int half = 0; half < 2; ++half) {
    const int c = c0 + half;
    if (c >= d.total_cols) break;
    int f = 0;
    while (f + 1 < d.nf && c >= d.colbase[f + 1]) ++f;
    const int r = c - d.colbase[f];
    const T* A = static_cast<const T*>(d.factors[f]);
    const int R = d.cols[f];
    const int32_t* tab = d.tables[f];
    T* dst = half == 0 ? &a[0].x : &a[0].y;
    // 8 rows per thread in flight (tall factors are latency-bound otherwise)
    const int64_t rows = d.rows[f];
    for (int64_t i0 = threadIdx.x; i0 < rows; i0 += 8 * (int64_t)blockDim.x) {
      int32_t e[8];
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int64_t i = i0 + (int64_t)u * blockDim.x;
        e[u] = i < rows ? tab[i] : 0;
        v[u] = i < rows ? A[i * R + r] : (T)0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (i0 + (int64_t)u * blockDim.x >= rows) break;
        const int bin = entry_bin(e[u]);
        if (bin >= m) continue;  // caller-supplied table outside [0, m): entry ignored
        atomicAdd(dst + 2 * (size_t)bin, entry_neg(e[u]) ? -v[u] : v[u]);
      }
    }
  }
  __syncthreads();
  const Cx<T>* F = fft_run<T>(a, b, plan, twp);
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const Cx<T> z = F[k];
    const Cx<T> zc = cconj(F[k == 0 ? 0 : m - k]);
    spectra[(size_t)c0 * m + k] = Cx<T>{(z.x + zc.x) * (T)0.5, (z.y + zc.y) * (T)0.5};
    if (c1 < d.total_cols) {
      const Cx<T> df = csub(z, zc);  // (z - conj z(-k)) / (2i)
      spectra[(size_t)c1 * m + k] = Cx<T>{df.y * (T)0.5, -df.x * (T)0.5};
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(512) k_factor_spectra(ChainDesc d, FftPlan plan,
                                                        const Cx<T>* __restrict__ tw,
                                                        Cx<T>* __restrict__ spectra) {
  pdl_trigger();
  pdl_wait();
  factor_spectra_body<T>(d, plan, tw, spectra, blockIdx.x);
}

// Block bx: Z columns 2 bx and 2 bx + 1 (column multi-index, factor 0 slowest).
template <typename T>
__device__ __forceinline__ void hadamard_ifft_body(const ChainDesc& d, int ncols,
                                                   const FftPlan& plan,
                                                   const Cx<T>* __restrict__ tw,
                                                   const Cx<T>* __restrict__ spectra,
                                                   T* __restrict__ Z, int bx,
                                                   __nv_bfloat16* __restrict__ Zb = nullptr,
                                                   int ldb = 0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = plan.m;
  Cx<T>* a = reinterpret_cast<Cx<T>*>(smem_raw);
  Cx<T>* b = a + m;
  const Cx<T>* twp = tw;
  if (plan.stage_tw) {
    Cx<T>* tws = b + m;
    for (int i = threadIdx.x; i < m; i += blockDim.x) tws[i] = tw[i];
    twp = tws;
  }
  const int c0 = 2 * bx;
  const bool has1 = c0 + 1 < ncols;
  int sp0[TS_MAX_ORDER], sp1[TS_MAX_ORDER];
  {
    int x0 = c0, x1 = c0 + 1;
    for (int f = d.nf - 1; f >= 0; --f) {
      sp0[f] = d.colbase[f] + x0 % d.cols[f];
      sp1[f] = d.colbase[f] + x1 % d.cols[f];
      x0 /= d.cols[f];
      x1 /= d.cols[f];
    }
  }
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    Cx<T> p0{1, 0}, p1{0, 0};
    if (has1) p1 = Cx<T>{1, 0};
    for (int f = 0; f < d.nf; ++f) {
      p0 = cmul(p0, spectra[(size_t)sp0[f] * m + k]);
      if (has1) p1 = cmul(p1, spectra[(size_t)sp1[f] * m + k]);
    }
    // inverse FFT of s = p0 + i p1 as conj(FFT(conj(s))) / m
    a[k] = Cx<T>{p0.x - p1.y, -(p0.y + p1.x)};
  }
  __syncthreads();
  const Cx<T>* F = fft_run<T>(a, b, plan, twp);
  const T inv_m = (T)1 / (T)m;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const T z0 = F[k].x * inv_m, z1 = -F[k].y * inv_m;
    Z[(size_t)c0 * m + k] = z0;
    if (has1) Z[(size_t)(c0 + 1) * m + k] = z1;
    if constexpr (sizeof(T) == 4) {
      if (Zb) {  // row c of Z^T in BF16 (the precision form's product operand)
        Zb[(size_t)c0 * ldb + k] = __float2bfloat16_rn((float)z0);
        if (has1) Zb[(size_t)(c0 + 1) * ldb + k] = __float2bfloat16_rn((float)z1);
      }
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(512) k_hadamard_ifft(ChainDesc d, int ncols, FftPlan plan,
                                                       const Cx<T>* __restrict__ tw,
                                                       const Cx<T>* __restrict__ spectra,
                                                       T* __restrict__ Z,
                                                       __nv_bfloat16* __restrict__ Zb, int ldb) {
  pdl_trigger();
  pdl_wait();
  hadamard_ifft_body<T>(d, ncols, plan, tw, spectra, Z, blockIdx.x, Zb, ldb);
}

// Many independent chains (one per blockIdx.y), each as in launch_ts_apply.
template <typename T>
__global__ void __launch_bounds__(512) k_factor_spectra_batched(const TsChainJob<T>* __restrict__ jobs) {
  const TsChainJob<T>& j = jobs[blockIdx.y];
  if ((int)blockIdx.x * 2 >= j.d.total_cols) return;
  factor_spectra_body<T>(j.d, j.plan, j.tw, j.spectra, blockIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(512) k_hadamard_ifft_batched(const TsChainJob<T>* __restrict__ jobs) {
  const TsChainJob<T>& j = jobs[blockIdx.y];
  if ((int)blockIdx.x * 2 >= j.ncols) return;
  hadamard_ifft_body<T>(j.d, j.ncols, j.plan, j.tw, j.spectra, j.Z, blockIdx.x);
}

// ---------------------------------------------------------------- adjoint of the chain

// Adjoint of Z = TensorSketch(chain) for a gradient dZ (column-major m x prod cols):
// column c of Z is the inverse FFT of prod_f U_f^(c_f) (U_f = CountSketch of factor f,
// ^ the DFT), so for real signals
//   dU_f[:, r] = IFFT( sum_{c : c_f = r} DFT(dZ[:, c]) * conj(prod_{j != f} U^_j[:, c_j]) )
// (a circular cross-correlation), and dA_f[i, r] = S_f(i) dU_f[H_f(i), r] (the transpose
// of the CountSketch: a hash/sign gather).

// Block bx: DFT of dZ columns 2 bx and 2 bx + 1 (one complex FFT of the pair).
template <typename T>
__global__ void __launch_bounds__(512) k_dz_spectra(int ncols, FftPlan plan,
                                                    const Cx<T>* __restrict__ tw,
                                                    const T* __restrict__ dZ,
                                                    Cx<T>* __restrict__ dspec) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = plan.m;
  Cx<T>* a = reinterpret_cast<Cx<T>*>(smem_raw);
  Cx<T>* b = a + m;
  const Cx<T>* twp = tw;
  if (plan.stage_tw) {
    Cx<T>* tws = b + m;
    for (int i = threadIdx.x; i < m; i += blockDim.x) tws[i] = tw[i];
    twp = tws;
  }
  const int c0 = 2 * blockIdx.x, c1 = c0 + 1;
  const bool has1 = c1 < ncols;
  for (int k = threadIdx.x; k < m; k += blockDim.x)
    a[k] = Cx<T>{dZ[(size_t)c0 * m + k], has1 ? dZ[(size_t)c1 * m + k] : (T)0};
  __syncthreads();
  const Cx<T>* F = fft_run<T>(a, b, plan, twp);
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    const Cx<T> z = F[k];
    const Cx<T> zc = cconj(F[k == 0 ? 0 : m - k]);
    dspec[(size_t)c0 * m + k] = Cx<T>{(z.x + zc.x) * (T)0.5, (z.y + zc.y) * (T)0.5};
    if (has1) {
      const Cx<T> df = csub(z, zc);
      dspec[(size_t)c1 * m + k] = Cx<T>{df.y * (T)0.5, -df.x * (T)0.5};
    }
  }
}

// Block bx: dU of flat factor columns 2 bx and 2 bx + 1 (real pair in one inverse FFT).
template <typename T>
__global__ void __launch_bounds__(512) k_adjoint_factor(ChainDesc d, FftPlan plan,
                                                        const Cx<T>* __restrict__ tw,
                                                        const Cx<T>* __restrict__ spectra,
                                                        const Cx<T>* __restrict__ dspec,
                                                        T* __restrict__ dU) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int m = plan.m;
  Cx<T>* a = reinterpret_cast<Cx<T>*>(smem_raw);
  Cx<T>* b = a + m;
  const Cx<T>* twp = tw;
  if (plan.stage_tw) {
    Cx<T>* tws = b + m;
    for (int i = threadIdx.x; i < m; i += blockDim.x) tws[i] = tw[i];
    twp = tws;
  }
  int fc[2], rc[2];
  bool has[2];
  for (int h = 0; h < 2; ++h) {
    const int c = 2 * blockIdx.x + h;
    has[h] = c < d.total_cols;
    int f = 0;
    while (has[h] && f + 1 < d.nf && c >= d.colbase[f + 1]) ++f;
    fc[h] = f;
    rc[h] = has[h] ? c - d.colbase[f] : 0;
  }
  // columns of Z: multi-index (c_0 .. c_{nf-1}), factor 0 slowest
  int ncols = 1;
  for (int f = 0; f < d.nf; ++f) ncols *= d.cols[f];
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    Cx<T> acc[2] = {Cx<T>{0, 0}, Cx<T>{0, 0}};
    for (int h = 0; h < 2; ++h) {
      if (!has[h]) continue;
      const int f = fc[h], r = rc[h];
      const int nother = ncols / d.cols[f];
      for (int o = 0; o < nother; ++o) {
        // multi-index with c_f = r and the others enumerated by o (C order)
        int rem = o, col = 0, stride = 1;
        Cx<T> p{1, 0};
        int cidx[TS_MAX_ORDER];
        for (int j = d.nf - 1; j >= 0; --j) {
          if (j == f) {
            cidx[j] = r;
          } else {
            cidx[j] = rem % d.cols[j];
            rem /= d.cols[j];
          }
        }
        for (int j = d.nf - 1; j >= 0; --j) {
          col += cidx[j] * stride;
          stride *= d.cols[j];
          if (j != f) p = cmul(p, spectra[(size_t)(d.colbase[j] + cidx[j]) * m + k]);
        }
        const Cx<T> g = dspec[(size_t)col * m + k];
        const Cx<T> t = cmul(g, cconj(p));
        acc[h].x += t.x;
        acc[h].y += t.y;
      }
    }
    // inverse FFT of s = acc0 + i acc1 as conj(FFT(conj(s))) / m
    a[k] = Cx<T>{acc[0].x - acc[1].y, -(acc[0].y + acc[1].x)};
  }
  __syncthreads();
  const Cx<T>* F = fft_run<T>(a, b, plan, twp);
  const T inv_m = (T)1 / (T)m;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    if (has[0]) dU[(size_t)(2 * blockIdx.x) * m + k] = F[k].x * inv_m;
    if (has[1]) dU[(size_t)(2 * blockIdx.x + 1) * m + k] = -F[k].y * inv_m;
  }
}

// dA_f[i, r] = S_f(i) dU[(colbase_f + r) m + H_f(i)] for every factor of the chain.
template <typename T>
struct GradOut {
  T* p[TS_MAX_ORDER];
};

template <typename T>
__global__ void k_adjoint_gather(ChainDesc d, int m, const T* __restrict__ dU, GradOut<T> grads) {
  const int f = blockIdx.y;
  if (f >= d.nf) return;
  const int R = d.cols[f];
  const int64_t total = d.rows[f] * R;
  T* g = grads.p[f];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / R;
    const int r = (int)(e - i * R);
    const int32_t t = d.tables[f][i];
    const int bin = entry_bin(t);
    T v = bin < m ? dU[(size_t)(d.colbase[f] + r) * m + bin] : (T)0;
    g[e] = entry_neg(t) ? -v : v;
  }
}

template <typename T>
ts_status launch_ts_adjoint(int nf, const int64_t* rows, const int* cols,
                            const int32_t* const* tables, int m, const Cx<T>* tw,
                            const Cx<T>* spectra, const T* dZ, Cx<T>* dspec, T* dU,
                            T* const* grads, cudaStream_t st) {
  ChainDesc d{};
  GradOut<T> go{};
  for (int f = 0; f < nf; ++f) go.p[f] = grads[f];
  d.nf = nf;
  int total = 0;
  long ncols = 1;
  int64_t maxrows = 0;
  for (int f = 0; f < nf; ++f) {
    d.rows[f] = rows[f];
    d.cols[f] = cols[f];
    d.colbase[f] = total;
    d.tables[f] = tables[f];
    total += cols[f];
    ncols *= cols[f];
    if (rows[f] * cols[f] > maxrows) maxrows = rows[f] * cols[f];
  }
  d.total_cols = total;
  FftPlan plan = make_fft_plan(m);
  plan.stage_tw = 3 * (size_t)m * sizeof(Cx<T>) <= kMaxSmem ? 1 : 0;
  const size_t smem = (2 + plan.stage_tw) * (size_t)m * sizeof(Cx<T>);
  TS_TRY(ensure_dynamic_smem((const void*)k_dz_spectra<T>, smem));
  TS_TRY(ensure_dynamic_smem((const void*)k_adjoint_factor<T>, smem));
  k_dz_spectra<T><<<ceil_div(ncols, 2), 512, smem, st>>>((int)ncols, plan, tw, dZ, dspec);
  TS_LAUNCH_CHECK();
  k_adjoint_factor<T><<<ceil_div(total, 2), 512, smem, st>>>(d, plan, tw, spectra, dspec, dU);
  TS_LAUNCH_CHECK();
  int blocks = ceil_div(maxrows, 256);
  if (blocks > 1024) blocks = 1024;
  k_adjoint_gather<T><<<dim3(blocks, nf), 256, 0, st>>>(d, m, dU, go);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

template <typename T>
TsChainJob<T> make_chain_job(int nf, const T* const* factors, const int64_t* rows,
                             const int* cols, const int32_t* const* tables, int m,
                             const Cx<T>* tw, Cx<T>* spectra, T* Z) {
  TsChainJob<T> j{};
  ChainDesc& d = j.d;
  d.nf = nf;
  int total = 0;
  long ncols = 1;
  for (int f = 0; f < nf; ++f) {
    d.factors[f] = factors[f];
    d.rows[f] = rows[f];
    d.cols[f] = cols[f];
    d.colbase[f] = total;
    d.tables[f] = tables[f];
    total += cols[f];
    ncols *= cols[f];
  }
  d.total_cols = total;
  j.ncols = (int)ncols;
  j.plan = make_fft_plan(m);
  j.plan.stage_tw = 3 * (size_t)m * sizeof(Cx<T>) <= kMaxSmem ? 1 : 0;
  j.tw = tw;
  j.spectra = spectra;
  j.Z = Z;
  return j;
}

template <typename T>
size_t chain_job_smem(const TsChainJob<T>& j) {
  return (2 + j.plan.stage_tw) * (size_t)j.plan.m * sizeof(Cx<T>);
}

template <typename T>
ts_status launch_ts_apply_batched(const TsChainJob<T>* jobs, int count, int max_spectra_blocks,
                                  int max_z_blocks, size_t smem, cudaStream_t st) {
  if (count < 1) return TS_OK;
  TS_TRY(ensure_dynamic_smem((const void*)k_factor_spectra_batched<T>, smem));
  TS_TRY(ensure_dynamic_smem((const void*)k_hadamard_ifft_batched<T>, smem));
  k_factor_spectra_batched<T><<<dim3(max_spectra_blocks, count), 512, smem, st>>>(jobs);
  TS_LAUNCH_CHECK();
  k_hadamard_ifft_batched<T><<<dim3(max_z_blocks, count), 512, smem, st>>>(jobs);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

template <typename T>
ts_status launch_ts_apply(int nf, const T* const* factors, const int64_t* rows, const int* cols,
                          const int32_t* const* tables, int m, const Cx<T>* tw, Cx<T>* spectra,
                          T* Z, cudaStream_t st, void* Zb_bf16, int ldb) {
  ChainDesc d{};
  d.nf = nf;
  int total = 0;
  long ncols = 1;
  for (int f = 0; f < nf; ++f) {
    d.factors[f] = factors[f];
    d.rows[f] = rows[f];
    d.cols[f] = cols[f];
    d.colbase[f] = total;
    d.tables[f] = tables[f];
    total += cols[f];
    ncols *= cols[f];
  }
  d.total_cols = total;
  FftPlan plan = make_fft_plan(m);
  plan.stage_tw = 3 * (size_t)m * sizeof(Cx<T>) <= kMaxSmem ? 1 : 0;
  const size_t smem = (2 + plan.stage_tw) * (size_t)m * sizeof(Cx<T>);
  TS_TRY(ensure_dynamic_smem((const void*)k_factor_spectra<T>, smem));
  TS_TRY(ensure_dynamic_smem((const void*)k_hadamard_ifft<T>, smem));
  TS_TRY(launch_pdl(k_factor_spectra<T>, dim3(ceil_div(total, 2)), dim3(512), smem, st, d, plan,
                    tw, spectra));
  TS_TRY(launch_pdl(k_hadamard_ifft<T>, dim3(ceil_div(ncols, 2)), dim3(512), smem, st, d,
                    (int)ncols, plan, tw, static_cast<const Cx<T>*>(spectra), Z,
                    static_cast<__nv_bfloat16*>(Zb_bf16), ldb));
  return TS_OK;
}

#define TS_INST_CHAIN(T)                                                                   \
  template TsChainJob<T> make_chain_job<T>(int, const T* const*, const int64_t*, const int*,   \
                                           const int32_t* const*, int, const Cx<T>*, Cx<T>*,  \
                                           T*);                                               \
  template size_t chain_job_smem<T>(const TsChainJob<T>&);                                     \
  template ts_status launch_ts_apply_batched<T>(const TsChainJob<T>*, int, int, int, size_t,   \
                                                cudaStream_t);
TS_INST_CHAIN(float)
TS_INST_CHAIN(double)
template ts_status launch_ts_adjoint<float>(int, const int64_t*, const int*,
                                            const int32_t* const*, int, const Cx<float>*,
                                            const Cx<float>*, const float*, Cx<float>*, float*,
                                            float* const*, cudaStream_t);
template ts_status launch_ts_adjoint<double>(int, const int64_t*, const int*,
                                             const int32_t* const*, int, const Cx<double>*,
                                             const Cx<double>*, const double*, Cx<double>*,
                                             double*, double* const*, cudaStream_t);
#undef TS_INST_CHAIN

template ts_status launch_twiddles<float>(int, Cx<float>*, cudaStream_t);
template ts_status launch_twiddles<double>(int, Cx<double>*, cudaStream_t);
template ts_status launch_ts_apply<float>(int, const float* const*, const int64_t*, const int*,
                                          const int32_t* const*, int, const Cx<float>*,
                                          Cx<float>*, float*, cudaStream_t, void*, int);
template ts_status launch_ts_apply<double>(int, const double* const*, const int64_t*, const int*,
                                           const int32_t* const*, int, const Cx<double>*,
                                           Cx<double>*, double*, cudaStream_t, void*, int);

}  // namespace ts

using namespace ts;

template <typename T>
static size_t ts_apply_scratch(int nf, const int32_t* cols, int m) {
  Bump b;
  int total = 0;
  for (int f = 0; f < nf; ++f) total += cols[f];
  b.take<Cx<T>>((size_t)m);
  b.take<Cx<T>>((size_t)m * total);
  return b.off;
}

extern "C" size_t tensorsketch_apply_scratch_bytes(int32_t nf, const int32_t* cols, int32_t m,
                                                   int32_t dtype) {
  if (nf < 1 || nf >= TS_MAX_ORDER || !cols || m < 1) return 0;
  return dtype == TS_F64 ? ts_apply_scratch<double>(nf, cols, m)
                         : ts_apply_scratch<float>(nf, cols, m);
}

template <typename T>
static ts_status ts_apply_impl(int nf, const void* const* factors, const int64_t* rows,
                               const int32_t* cols, const int32_t* const* tables, int m, void* Z,
                               void* scratch, cudaStream_t st) {
  Bump b{static_cast<char*>(scratch)};
  int total = 0;
  for (int f = 0; f < nf; ++f) total += cols[f];
  Cx<T>* tw = b.take<Cx<T>>((size_t)m);
  Cx<T>* spectra = b.take<Cx<T>>((size_t)m * total);
  const T* fp[TS_MAX_ORDER];
  int c[TS_MAX_ORDER];
  for (int f = 0; f < nf; ++f) {
    fp[f] = static_cast<const T*>(factors[f]);
    c[f] = cols[f];
  }
  TS_TRY(launch_twiddles<T>(m, tw, st));
  return launch_ts_apply<T>(nf, fp, rows, c, tables, m, tw, spectra, static_cast<T*>(Z), st);
}

extern "C" ts_status tensorsketch_apply(int32_t nf, const void* const* factors,
                                        const int64_t* rows, const int32_t* cols,
                                        const int32_t* const* tables, int32_t m, int32_t dtype,
                                        void* Z_out, void* scratch, size_t scratch_bytes,
                                        ts_stream stream) {
  clear_error();
  if (!factors || !rows || !cols || !tables || !Z_out)
    return fail(TS_ERR_INVALID_ARG, "tensorsketch_apply: NULL argument");
  if (dtype != TS_F32 && dtype != TS_F64)
    return fail(TS_ERR_INVALID_ARG, "tensorsketch_apply: bad dtype %d", dtype);
  if (nf < 1 || nf >= TS_MAX_ORDER)
    return fail(TS_ERR_SHAPE, "tensorsketch_apply: nf=%d outside [1,%d)", nf, TS_MAX_ORDER);
  const int maxlen = dtype == TS_F64 ? fft_max_len<double>() : fft_max_len<float>();
  if (m < 2 || m > maxlen)
    return fail(TS_ERR_SHAPE, "tensorsketch_apply: m=%d outside [2,%d]", m, maxlen);
  long ncols = 1;
  for (int f = 0; f < nf; ++f) {
    if (!factors[f] || !tables[f] || rows[f] < 1 || cols[f] < 1)
      return fail(TS_ERR_INVALID_ARG, "tensorsketch_apply: bad factor %d", f);
    ncols *= cols[f];
  }
  if (ncols > (1l << 24)) return fail(TS_ERR_SHAPE, "tensorsketch_apply: too many columns");
  const size_t need = tensorsketch_apply_scratch_bytes(nf, cols, m, dtype);
  if (!scratch || scratch_bytes < need || ((uintptr_t)scratch & 255))
    return fail(TS_ERR_WORKSPACE, "tensorsketch_apply: need %zu bytes of 256-aligned scratch",
                need);
  cudaStream_t st = (cudaStream_t)stream;
  return dtype == TS_F64
             ? ts_apply_impl<double>(nf, factors, rows, cols, tables, m, Z_out, scratch, st)
             : ts_apply_impl<float>(nf, factors, rows, cols, tables, m, Z_out, scratch, st);
}
