// Host orchestration of Sketch-Tucker-ALS (Alg. 4) and the C-ABI entry points
// that compose the kernels: Init-RRF (Alg. 3), the sketched subproblem solve
// (Alg. 5 / exact), the leverage-score sketch, the fitness, the driver itself and
// CP-Sketch-Tucker (Alg. 6).  Every step runs on the caller's stream in the
// caller's scratch; the host only validates, carves the workspace and enqueues.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"

namespace ts {

// ---------------------------------------------------------------- validation

static ts_status check_tensor(const ts_tensor* X, const char* who) {
  if (!X) return fail(TS_ERR_INVALID_ARG, "%s: tensor is NULL", who);
  if (X->order < 2 || X->order > TS_MAX_ORDER)
    return fail(TS_ERR_SHAPE, "%s: order %d outside [2,%d]", who, X->order, TS_MAX_ORDER);
  if (X->dtype != TS_F32 && X->dtype != TS_F64)
    return fail(TS_ERR_INVALID_ARG, "%s: bad dtype %d", who, X->dtype);
  if (X->format != TS_DENSE && X->format != TS_COO)
    return fail(TS_ERR_INVALID_ARG, "%s: bad format %d", who, X->format);
  for (int k = 0; k < X->order; ++k)
    if (X->dims[k] < 1 || X->dims[k] >= (int64_t)kP31)
      return fail(TS_ERR_SHAPE, "%s: dims[%d]=%lld outside [1, 2^31-1)", who, k,
                  (long long)X->dims[k]);
  if (X->format == TS_COO) {
    if (X->nnz < 0) return fail(TS_ERR_INVALID_ARG, "%s: nnz < 0", who);
    if (X->nnz > 0 && (!X->indices || !X->values))
      return fail(TS_ERR_INVALID_ARG, "%s: COO arrays are NULL", who);
  } else if (!X->values) {
    return fail(TS_ERR_INVALID_ARG, "%s: values is NULL", who);
  }
  return TS_OK;
}

static int64_t prod_other(const int64_t* d, int N, int n) {
  int64_t p = 1;
  for (int k = 0; k < N; ++k)
    if (k != n) p *= d[k];
  return p;
}

static void rrf_widths(const ts_tensor& X, int n, int R, int m, int k1_opt, int k2_opt, int* k1o,
                       int* k2o) {
  const int64_t K = prod_other(X.dims, X.order, n);
  long k1 = k1_opt > 0 ? k1_opt : (long)ceil(sqrt((double)m));
  long k2 = k2_opt > 0 ? k2_opt : (long)R * R + k1;
  if (k2 > K) k2 = K;
  long k1c = k1 < k2 ? k1 : k2;
  if (k1c > X.dims[n]) k1c = X.dims[n];
  if (k1c < R) k1c = R;
  *k1o = (int)k1c;
  *k2o = (int)k2;
}

// The fused single-block solve applies when Z^T Y (r x s) is small enough to form
// and the block's shared-memory layout fits.
static bool fused_ok(int r, long s, int kc, int R, int solve, size_t tsize, bool fp64) {
  if ((long)r * s > (1l << 22)) return false;
  return lrls_fused_supported(r, (int)s, kc, R, solve, tsize, fp64);
}

static int rsvd_width(int R, int p, int r, int64_t s) {
  long k = R + p;
  if (k > r) k = r;
  if (k > s) k = s;
  return (int)(k < R ? R : k);
}

struct Shape {
  int N;
  int m;
  int sweeps;
  int kind;
  int solve;
  int oversample;
  bool rrf;
  bool fp64solve;  // FP64 QR / polish on FP32 data
  bool bf16gram;   // [G | W | H] on the tensor cores in BF16 (FP32 data, fused subproblems)
  bool coo_lev;    // leverage sampling of a COO tensor: per-mode fibre indices
  int ranks[TS_MAX_ORDER];
  int r[TS_MAX_ORDER];   // prod_{k != n} ranks[k]
  int kc[TS_MAX_ORDER];  // RSVD width of subproblem n
  bool fused[TS_MAX_ORDER];  // subproblem n takes the fused single-block solve
  bool large[TS_MAX_ORDER];  // subproblem n inverts Z^T Z by Newton-Schulz (large r)
  int k1[TS_MAX_ORDER], k2[TS_MAX_ORDER];
  OmegaBlocks ob;                 // every Omega(sweep, n): mode blocks s_n x (sweeps k_n)
  int64_t yom_off[TS_MAX_ORDER];  // Y_n Omega(., n): mode blocks m x (sweeps k_n)
  int64_t yom_total;
  int64_t smax;
  int rmax, kmax, Rmax, k1max, k2max, chain_cols_max;
};

static ts_status plan_shape(const ts_tensor* X, const int32_t* ranks, int kind, int m, int sweeps,
                            const ts_options* opt, bool want_residual, Shape& S) {
  TS_TRY(check_tensor(X, "tucker_als_sketched"));
  if (!ranks || !opt) return fail(TS_ERR_INVALID_ARG, "tucker_als_sketched: NULL ranks/options");
  if (kind != TS_TENSORSKETCH && kind != TS_LEVERAGE && kind != TS_LEVERAGE_DET)
    return fail(TS_ERR_INVALID_ARG, "tucker_als_sketched: bad sketch kind %d", kind);
  if (opt->solve != TS_SOLVE_RSVD && opt->solve != TS_SOLVE_EXACT)
    return fail(TS_ERR_INVALID_ARG, "tucker_als_sketched: bad solve kind %d", opt->solve);
  if (sweeps < 1) return fail(TS_ERR_SHAPE, "tucker_als_sketched: sweeps %d < 1", sweeps);
  if (kind != TS_TENSORSKETCH && X->format == TS_COO) {
    if (X->nnz >= (int64_t(1) << 30))
      return fail(TS_ERR_UNSUPPORTED,
                  "tucker_als_sketched: leverage sampling of COO tensors takes < 2^30 nonzeros");
    for (int n = 0; n < X->order; ++n) {
      if (!fibre_keys_fit(*X, n))
        return fail(TS_ERR_UNSUPPORTED,
                    "tucker_als_sketched: fibre keys of mode %d exceed 64 bits", n);
      if (kind == TS_LEVERAGE_DET && leverage_det_candidates(*X, n) < 0)
        return fail(TS_ERR_UNSUPPORTED,
                    "tucker_als_sketched: deterministic leverage over more than 2^31 rows");
    }
  }
  if (kind == TS_LEVERAGE_DET && X->format == TS_DENSE)
    for (int n = 0; n < X->order; ++n)
      if (leverage_det_candidates(*X, n) < 0)
        return fail(TS_ERR_UNSUPPORTED,
                    "tucker_als_sketched: deterministic leverage over more than 2^31 rows");
  if (want_residual && X->format == TS_COO &&
      (!fit_coo_supported(*X) || !fit_coo_model_ok(*X, ranks)))
    return fail(TS_ERR_UNSUPPORTED,
                "tucker_als_sketched: COO residual needs < 2^30 nonzeros, fibre keys of the "
                "largest mode within 64 bits, a core <= 200 KB and a last rank <= 64");
  S.N = X->order;
  S.m = m;
  S.sweeps = sweeps;
  S.kind = kind;
  S.solve = opt->solve;
  S.oversample = opt->rsvd_oversample < 0 ? 5 : opt->rsvd_oversample;
  S.rrf = !opt->init_given;
  S.fp64solve = opt->solve_fp64 != 0 && X->dtype == TS_F32;
  S.bf16gram = opt->gram_bf16 != 0 && X->dtype == TS_F32;
  S.coo_lev = kind != TS_TENSORSKETCH && X->format == TS_COO;
  S.smax = 0;
  S.rmax = S.kmax = S.Rmax = S.k1max = S.k2max = S.chain_cols_max = 0;
  memset(&S.ob, 0, sizeof(S.ob));
  S.ob.N = S.N;
  S.ob.nsweeps = sweeps;
  S.yom_total = 0;
  const size_t tsz = dtype_size(X->dtype);
  for (int k = 0; k < S.N; ++k) {
    if (ranks[k] < 1 || ranks[k] >= X->dims[k])
      return fail(TS_ERR_SHAPE, "tucker_als_sketched: rank[%d]=%d must lie in [1, dims[%d]=%lld)",
                  k, ranks[k], k, (long long)X->dims[k]);
    S.ranks[k] = ranks[k];
    if (X->dims[k] > S.smax) S.smax = X->dims[k];
    if (ranks[k] > S.Rmax) S.Rmax = ranks[k];
  }
  const int fftmax = X->dtype == TS_F64 ? fft_max_len<double>() : fft_max_len<float>();
  if (kind == TS_TENSORSKETCH && (m < 2 || m > fftmax))
    return fail(TS_ERR_SHAPE, "tucker_als_sketched: m=%d outside [2,%d]", m, fftmax);
  if (m < 1) return fail(TS_ERR_SHAPE, "tucker_als_sketched: m < 1");
  for (int n = 0; n < S.N; ++n) {
    long r = 1;
    int cc = 0;
    for (int k = 0; k < S.N; ++k)
      if (k != n) {
        r *= ranks[k];
        cc += ranks[k];
      }
    if (r > m)
      return fail(TS_ERR_SHAPE,
                  "tucker_als_sketched: m=%d < prod of the other ranks (%ld) for mode %d", m, r, n);
    S.r[n] = (int)r;
    S.kc[n] = rsvd_width(ranks[n], S.oversample, (int)r, X->dims[n]);
    S.fused[n] = fused_ok((int)r, X->dims[n], S.kc[n], ranks[n], S.solve, tsz, S.fp64solve);
    S.large[n] = false;
    if (S.fused[n]) {
      // the fused block solve covers this subproblem
    } else if (S.solve == TS_SOLVE_RSVD) {
      if (S.kc[n] > kMaxEig)
        return fail(TS_ERR_SHAPE, "tucker_als_sketched: RSVD width %d > %d", S.kc[n], kMaxEig);
      if (rsvd_stage1_smem_bytes((int)r, S.kc[n], tsz, S.fp64solve) > kMaxSmem) {
        // G^{-1} by Newton-Schulz products, QR in one block
        if (qr_only_smem_bytes((int)r, S.kc[n], S.fp64solve, tsz) > kMaxSmem)
          return fail(TS_ERR_UNSUPPORTED,
                      "tucker_als_sketched: r=%ld, k=%d too large for the RSVD solve", r,
                      S.kc[n]);
        S.large[n] = true;
      }
    } else {
      if (r > kMaxEig || chol_solve_smem_bytes((int)r, tsz) > kMaxSmem)
        return fail(TS_ERR_UNSUPPORTED, "tucker_als_sketched: r=%ld > %d for the exact solve", r,
                    kMaxEig);
    }
    if (r > S.rmax) S.rmax = (int)r;
    if (S.kc[n] > S.kmax) S.kmax = S.kc[n];
    if (cc > S.chain_cols_max) S.chain_cols_max = cc;
    S.ob.rows[n] = X->dims[n];
    S.ob.k[n] = S.kc[n];
    S.ob.off[n] = S.ob.total;
    S.ob.total += X->dims[n] * (int64_t)sweeps * S.kc[n];
    S.yom_off[n] = S.yom_total;
    S.yom_total += (int64_t)m * sweeps * S.kc[n];
    S.k1[n] = S.k2[n] = 0;
    if (S.rrf && n >= 1) {
      rrf_widths(*X, n, ranks[n], m, opt->rrf_k1, opt->rrf_k2, &S.k1[n], &S.k2[n]);
      if (S.k1[n] > kMaxEig)
        return fail(TS_ERR_SHAPE, "tucker_als_sketched: RRF width k1=%d > %d", S.k1[n], kMaxEig);
      if (S.k1[n] > S.k1max) S.k1max = S.k1[n];
      if (S.k2[n] > S.k2max) S.k2max = S.k2[n];
    }
  }
  return TS_OK;
}

// ---------------------------------------------------------------- workspace

template <typename T>
struct Work {
  int* flag;
  unsigned* counters;
  GemmSplit<T> split;
  int32_t* tab[TS_MAX_ORDER][TS_MAX_ORDER];
  int32_t* rtab[TS_MAX_ORDER][TS_MAX_ORDER];
  T* Y[TS_MAX_ORDER];
  T* Wt[TS_MAX_ORDER];
  Cx<T>* tw;
  Cx<T>* spectra;
  T* ZW;   // column-major m x (r + k): Z, then Y Omega
  T* GW;   // [Z^T Z | Z^T Y Omega] (r x (r + k)) or [Z^T Z | Z^T Y] (r x (r + s), fused path)
  T* Mbuf; // fused path: D (k x s) or X (r x s)
  T *Ginv, *NS1, *NS2, *Cb;  // large-r path: G^{-1}, Newton-Schulz scratch, C = G^{-1} W
  T* Om;   // Omega of every (sweep, mode): mode blocks s_n x (sweeps k_n)
  T* YOm;  // Y_n Omega(sweep, n) for every (sweep, mode): mode blocks m x (sweeps k_n)
  T *Q, *E, *Mm, *D, *K, *CnT, *Fm, *H, *Xs, *Gm, *Bm, *Ylev;
  int32_t* samples;
  double* levscr;
  FibreIndex fib[TS_MAX_ORDER];  // COO leverage sampling: mode-n fibre indices
  T* fitQ;
  double* fitacc;
  FitCooWork fitc;  // COO residual
  void* Bt[TS_MAX_ORDER];  // BF16 precision form: [Z | Y Omega | Y]^T per mode and sweep
  size_t bt_stride[TS_MAX_ORDER];  // bytes between consecutive sweeps' operands
  float* gpart;            // its split-K partial sums
};

// Rows of the BF16 operand [Z | Y Omega | Y]^T of subproblem n (exact solve: [Z | Y]^T).
static int bf16_cols(const Shape& S, int n, int s) {
  return S.r[n] + (S.solve == TS_SOLVE_RSVD ? S.kc[n] : 0) + s;
}

template <typename T>
static void carve(const ts_tensor& X, const Shape& S, bool want_residual, Bump& b, Work<T>& w) {
  memset(&w, 0, sizeof(w));
  const int N = S.N, m = S.m;
  w.flag = b.take<int>(64);
  w.counters = b.take<unsigned>(kGemmCounters);
  if (S.kind == TS_TENSORSKETCH) {
    for (int n = 0; n < N; ++n)
      for (int k = 0; k < N; ++k)
        if (k != n) w.tab[n][k] = b.take<int32_t>((size_t)X.dims[k]);
    for (int n = 0; n < N; ++n) w.Y[n] = b.take<T>((size_t)m * X.dims[n]);
    w.tw = b.take<Cx<T>>((size_t)m);
    w.spectra = b.take<Cx<T>>((size_t)m * S.chain_cols_max);
  }
  if (S.rrf) {
    for (int n = 1; n < N; ++n) {
      for (int k = 0; k < N; ++k)
        if (k != n) w.rtab[n][k] = b.take<int32_t>((size_t)X.dims[k]);
      w.Wt[n] = b.take<T>((size_t)S.k2[n] * X.dims[n]);
    }
    w.Gm = b.take<T>((size_t)S.k2max * S.k1max);
    w.Bm = b.take<T>((size_t)S.smax * S.k1max);
  }
  const int r = S.rmax, k = S.kmax, R = S.Rmax;
  const int64_t s = S.smax;
  int eign = k;
  if (S.solve == TS_SOLVE_EXACT && r > eign) eign = r;
  if (S.k1max > eign) eign = S.k1max;
  size_t gw = (size_t)r * (r + k), mb = 0;
  for (int n = 0; n < N; ++n)
    if (S.fused[n]) {
      const size_t h = (size_t)S.r[n] * (S.r[n] + S.kc[n] + X.dims[n]);
      const size_t nn = S.solve == TS_SOLVE_RSVD ? S.kc[n] : S.r[n];
      if (h > gw) gw = h;
      if (nn * X.dims[n] > mb) mb = nn * X.dims[n];
    }
  w.ZW = b.take<T>((size_t)m * (r + k));
  w.GW = b.take<T>(gw);
  w.Mbuf = b.take<T>(mb);
  bool any_large = false;
  for (int n = 0; n < N; ++n) any_large |= S.large[n];
  if (any_large) {
    w.Ginv = b.take<T>((size_t)r * r);
    w.NS1 = b.take<T>(2 * (size_t)r * r);
    w.NS2 = b.take<T>((size_t)r * r);
    w.Cb = b.take<T>((size_t)r * k);
  }
  if (S.solve == TS_SOLVE_RSVD) {
    w.Om = b.take<T>((size_t)S.ob.total);
    if (S.kind == TS_TENSORSKETCH) w.YOm = b.take<T>((size_t)S.yom_total);
  }
  w.Q = b.take<T>((size_t)r * k);
  w.E = b.take<T>((size_t)r * k);
  w.Mm = b.take<T>((size_t)m * k);
  w.D = b.take<T>((size_t)k * s);
  w.K = b.take<T>((size_t)eign * eign);
  w.CnT = b.take<T>((size_t)r * R);
  w.Fm = b.take<T>((size_t)eign * R);
  if (S.solve == TS_SOLVE_EXACT) {
    w.H = b.take<T>((size_t)r * s);
    w.Xs = b.take<T>((size_t)r * s);
  }
  if (S.kind != TS_TENSORSKETCH) {
    w.Ylev = b.take<T>((size_t)m * s);
    w.samples = b.take<int32_t>((size_t)m * (N - 1));
    size_t lv = 0;
    for (int n = 0; n < N; ++n) {
      size_t t = leverage_scratch_doubles(X, n, m);
      if (t > lv) lv = t;
    }
    w.levscr = b.take<double>(lv);
    if (S.coo_lev)
      for (int n = 0; n < N; ++n) w.fib[n] = fibre_index_carve(X, n, b);
  }
  size_t pm = (size_t)r * (r + k);
  const size_t cands[] = {(size_t)m * k, (size_t)k * s, (size_t)eign * eign, (size_t)s * S.k1max,
                          S.solve == TS_SOLVE_EXACT ? (size_t)r * s : 0};
  for (size_t c : cands)
    if (c > pm) pm = c;
  w.split.partial_elems = 32 * pm;
  w.split.partial = b.take<T>(w.split.partial_elems);
  w.split.counters = w.counters;
  w.split.ncounters = kGemmCounters;
  if (want_residual && X.format == TS_DENSE) {
    w.fitQ = b.take<T>(fit_dense_scratch_elems<T>(X, S.ranks));
    w.fitacc = b.take<double>(2);
  }
  if (want_residual && X.format == TS_COO) w.fitc = fit_coo_carve(X, S.ranks, b);
  if (S.bf16gram) {
    size_t part = 0;
    for (int n = 0; n < N; ++n) {
      if (!S.fused[n]) continue;
      const int cols = bf16_cols(S, n, (int)X.dims[n]);
      w.bt_stride[n] = (size_t)cols * gram_tc_ld(m) * 2;
      w.Bt[n] = b.take<uint16_t>((size_t)cols * gram_tc_ld(m) * S.sweeps);
      const size_t p = gram_tc_partial_elems(S.r[n], cols, m);
      if (p > part) part = p;
    }
    w.gpart = b.take<float>(part);
  }
}

// ---------------------------------------------------------------- building blocks

template <typename T>
static MatView<T> mv(const T* p, long rs, long cs) {
  return MatView<T>{p, rs, cs};
}
template <typename T>
static OutView<T> ov(T* p, long rs, long cs) {
  return OutView<T>{p, rs, cs};
}

// The BF16 operand of one subproblem: rows [0, r) Z^T, then (Y Omega)^T, then Y^T;
// prefilled: Z^T (written by the inverse FFT), (Y Omega)^T and Y^T (written once per pass
// over T) are already in place.
struct Bf16Op {
  void* Bt;
  bool prefilled;
};

// Sketched subproblem on Z = ZW[:, :r] (column-major) and Y (m x s) -> CnT (r x R),
// A_out (s x R), core scattered when core != null.  RSVD (Alg. 5): yom views Y Omega
// (m x k) when the caller formed it, else it is formed here from the test matrix Om
// (s x k, row stride ldo) into ZW[:, r:r+k].  Exact: the truncated solve of Theorem 4.1.
template <typename T>
static ts_status solve_subproblem(int m, int r, int s, int R, int solve, int kc, bool fp64,
                                  const T* Om, long ldo, const MatView<T>* yom, const T* Y,
                                  Work<T>& w, T* A_out, T* core, const CoreMap& map,
                                  cudaStream_t st, const Bf16Op* bf = nullptr) {
  T* ZW = w.ZW;
  const MatView<T> Zt = mv<T>(ZW, m, 1);  // r x m view of Z^T
  const MatView<T> Zm = mv<T>(ZW, 1, m);  // m x r view of Z
  const GemmSplit<T>* sp = &w.split;
  const int k = kc;
  MatView<T> yv{};
  if (solve == TS_SOLVE_RSVD) {
    if (yom) {
      yv = *yom;
    } else {
      if (s >= kTallMinS)
        TS_TRY(wide_nn<T>(m, k, s, Y, s, Om, ldo, ZW + (size_t)r * m, 1, m, sp->partial,
                          sp->partial_elems, st));
      else
        TS_TRY(gemm<T>(m, k, s, 1.0, mv<T>(Y, s, 1), mv<T>(Om, ldo, 1), 0.0,
                       ov<T>(ZW + (size_t)r * m, 1, m), sp, st));
      yv = mv<T>(ZW + (size_t)r * m, 1, m);
    }
  }
  if (fused_ok(r, s, kc, R, solve, sizeof(T), fp64)) {
    // [G | W | H] = Z^T [Z | Y Omega | Y] (exact: [G | H]) in one product, then the whole
    // solve in one block
    if constexpr (sizeof(T) == 4) {
      if (bf) {  // BF16 precision form of the product, on the tensor cores
        const int kk = solve == TS_SOLVE_RSVD ? k : 0;
        const int N = r + kk + s;
        char* bt = static_cast<char*>(bf->Bt);
        const size_t row = 2 * (size_t)gram_tc_ld(m);
        if (!bf->prefilled) {
          TS_TRY(pack_bf16(ZW, m, 1, r, m, bt, st));  // Z^T: Z is column-major
          if (kk) TS_TRY(pack_bf16(yv.p, yv.cs, yv.rs, kk, m, bt + r * row, st));
          TS_TRY(pack_bf16(Y, 1, s, s, m, bt + (size_t)(r + kk) * row, st));
        }
        CUtensorMap ma, mb;
        TS_TRY(gram_tc_map(bt, r, m, &ma));
        TS_TRY(gram_tc_map(bt, N, m, &mb));
        TS_TRY(gram_tc(ma, mb, r, N, m, w.GW, N, w.gpart, w.flag, st));
        return launch_lrls_fused<T>(r, s, k, R, solve, fp64, w.GW, N, kk ? w.GW + r : nullptr,
                                    N, w.GW + r + kk, N, w.Mbuf, w.CnT, A_out, core, map,
                                    w.flag, st);
      }
    }
    if (solve == TS_SOLVE_RSVD) {
      const int N = r + k + s;
      TS_TRY(gemm3<T>(r, N, m, 1.0, Zt, Zm, r, yv, r + k, mv<T>(Y, s, 1), 0.0,
                      ov<T>(w.GW, N, 1), sp, st));
      return launch_lrls_fused<T>(r, s, k, R, solve, fp64, w.GW, N, w.GW + r, N, w.GW + r + k,
                                  N, w.Mbuf, w.CnT, A_out, core, map, w.flag, st);
    }
    const int N = r + s;
    TS_TRY(gemm2<T>(r, N, m, 1.0, Zt, Zm, r, mv<T>(Y, s, 1), 0.0, ov<T>(w.GW, N, 1), sp, st));
    return launch_lrls_fused<T>(r, s, k, R, solve, fp64, w.GW, N, nullptr, 0, w.GW + r, N,
                                w.Mbuf, w.CnT, A_out, core, map, w.flag, st);
  }
  if (solve == TS_SOLVE_RSVD) {
    // [G | W] = Z^T [Z | Y Omega] in one product
    TS_TRY(gemm3<T>(r, r + k, m, 1.0, Zt, Zm, r, yv, r + k, yv, 0.0, ov<T>(w.GW, r + k, 1), sp,
                    st));
    if (rsvd_stage1_smem_bytes(r, k, sizeof(T), fp64) <= kMaxSmem) {
      TS_TRY(launch_rsvd_stage1<T>(r, k, w.GW, r + k, w.GW + r, r + k, w.Q, w.E, fp64, w.flag,
                                   st));
    } else {
      // G^{-1} by Newton-Schulz; C = G^{-1} W; Q = qr(C); E = G^{-1} Q
      TS_TRY(newton_schulz_inverse<T>(r, w.GW, r + k, w.Ginv, w.NS1, w.NS2, kNewtonSchulzIters,
                                      w.flag + 8,
                                      sp, st));
      TS_TRY(gemm<T>(r, k, r, 1.0, mv<T>(w.Ginv, r, 1), mv<T>(w.GW + r, r + k, 1), 0.0,
                     ov<T>(w.Cb, k, 1), sp, st));
      TS_TRY(launch_qr_only<T>(r, k, w.Cb, w.Q, fp64, st));
      TS_TRY(gemm<T>(r, k, r, 1.0, mv<T>(w.Ginv, r, 1), mv<T>(w.Q, k, 1), 0.0, ov<T>(w.E, k, 1),
                     sp, st));
    }
    // M = Z E (m x k);  D = M^T Y (k x s);  K = D D^T (k x k)
    TS_TRY(gemm<T>(m, k, r, 1.0, Zm, mv<T>(w.E, k, 1), 0.0, ov<T>(w.Mm, k, 1), sp, st));
    if (s >= kTallMinS)
      TS_TRY(tall_tn<T>(m, k, s, w.Mm, k, Y, s, w.D, s, sp->partial, sp->partial_elems, st));
    else
      TS_TRY(gemm<T>(k, s, m, 1.0, mv<T>(w.Mm, 1, k), mv<T>(Y, s, 1), 0.0, ov<T>(w.D, s, 1), sp,
                     st));
    if (s >= kTallMinS)
      TS_TRY(gram_wide<T>(k, s, w.D, s, w.K, k, sp->partial, sp->partial_elems, st));
    else
      TS_TRY(gemm<T>(k, k, s, 1.0, mv<T>(w.D, s, 1), mv<T>(w.D, 1, s), 0.0, ov<T>(w.K, k, 1), sp,
                     st));
    TS_TRY(launch_eig_small<T>(k, R, w.K, w.Q, r, w.CnT, w.Fm, nullptr, fp64, w.flag, st));
    // A = D^T Fm, signed; core written
    return launch_finalize<T>(s, R, w.D, 1, s, k, w.Fm, A_out, w.CnT, r, core, map, st,
                              w.split.partial, w.split.partial_elems * sizeof(T));
  }
  // exact: G = Z^T Z;  H = Z^T Y;  X = G^{-1} H;  K = X X^T;  A = X^T Fm
  TS_TRY(gemm<T>(r, r, m, 1.0, Zt, Zm, 0.0, ov<T>(w.GW, r, 1), sp, st));
  TS_TRY(gemm<T>(r, s, m, 1.0, Zt, mv<T>(Y, s, 1), 0.0, ov<T>(w.H, s, 1), sp, st));
  TS_TRY(launch_chol_solve<T>(r, s, w.GW, w.H, w.Xs, w.flag, st));
  TS_TRY(gemm<T>(r, r, s, 1.0, mv<T>(w.Xs, s, 1), mv<T>(w.Xs, 1, s), 0.0, ov<T>(w.K, r, 1), sp,
                 st));
  TS_TRY(launch_eig_small<T>(r, R, w.K, nullptr, r, w.CnT, w.Fm, nullptr, fp64, w.flag, st));
  return launch_finalize<T>(s, R, w.Xs, 1, s, r, w.Fm, A_out, w.CnT, r, core, map, st,
                            w.split.partial, w.split.partial_elems * sizeof(T));
}

template <typename T>
static ts_status build_ts_tables(const ts_tensor& X, const Shape& S, uint64_t seed, int sweep,
                                 Work<T>& w, cudaStream_t st) {
  for (int n = 0; n < S.N; ++n)
    for (int k = 0; k < S.N; ++k)
      if (k != n)
        TS_TRY(launch_hash_table(seed, TS_PURPOSE_TS_HASH, sweep, n, k, X.dims[k], S.m,
                                 w.tab[n][k], st));
  return TS_OK;
}

template <typename T>
static ts_status sketch_rhs_all(const ts_tensor& X, const Shape& S, Work<T>& w, cudaStream_t st) {
  SketchJob jobs[kMaxJobs];
  for (int n = 0; n < S.N; ++n) {
    jobs[n].mode = n;
    jobs[n].nbins = S.m;
    jobs[n].out = w.Y[n];
    for (int k = 0; k < S.N; ++k) jobs[n].tables[k] = w.tab[n][k];
  }
  return launch_input_sketch<T>(X, jobs, S.N, w.flag, st);
}

// Init-RRF (Alg. 3) for every mode n >= 1: one pass over X for all CountSketch
// factors, then per mode B = W^T G, B^T B = V Lambda V^T, U = B V Sigma^{-1}.
template <typename T>
static ts_status rrf_all(const ts_tensor& X, const Shape& S, uint64_t seed, Work<T>& w,
                         T* const* factors, cudaStream_t st) {
  SketchJob jobs[kMaxJobs];
  int nj = 0;
  for (int n = 1; n < S.N; ++n) {
    for (int k = 0; k < S.N; ++k)
      if (k != n)
        TS_TRY(launch_hash_table(seed, TS_PURPOSE_RRF_HASH, 0, n, k, X.dims[k], S.k2[n],
                                 w.rtab[n][k], st));
    jobs[nj].mode = n;
    jobs[nj].nbins = S.k2[n];
    jobs[nj].out = w.Wt[n];
    for (int k = 0; k < S.N; ++k) jobs[nj].tables[k] = w.rtab[n][k];
    ++nj;
  }
  TS_TRY(launch_input_sketch<T>(X, jobs, nj, w.flag, st));
  CoreMap none{};
  for (int n = 1; n < S.N; ++n) {
    const int k1 = S.k1[n], k2 = S.k2[n], R = S.ranks[n];
    const int s = (int)X.dims[n];
    TS_TRY(launch_gaussian<T>(seed, make_tag(TS_PURPOSE_RRF_GAUSS, 0, n, 0), (int64_t)k2 * k1,
                              1.0 / sqrt((double)k1), w.Gm, st));
    TS_TRY(gemm<T>(s, k1, k2, 1.0, mv<T>(w.Wt[n], 1, s), mv<T>(w.Gm, k1, 1), 0.0,
                   ov<T>(w.Bm, k1, 1), &w.split, st));
    TS_TRY(gemm<T>(k1, k1, s, 1.0, mv<T>(w.Bm, 1, k1), mv<T>(w.Bm, k1, 1), 0.0, ov<T>(w.K, k1, 1),
                   &w.split, st));
    TS_TRY(launch_eig_small<T>(k1, R, w.K, nullptr, k1, nullptr, w.Fm, nullptr, S.fp64solve,
                               w.flag, st));
    TS_TRY(launch_finalize<T>(s, R, w.Bm, k1, 1, k1, w.Fm, factors[n], nullptr, 0, nullptr, none,
                              st, w.split.partial, w.split.partial_elems * sizeof(T)));
  }
  return TS_OK;
}

// BF16 precision form: Y_n^T into the last s_n rows of each mode's operand, once per
// pass over T (the sketches are fixed between passes).
template <typename T>
static ts_status pack_rhs_bf16(const ts_tensor& X, const Shape& S, Work<T>& w, int t0, int nt,
                               cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (!S.bf16gram || S.kind != TS_TENSORSKETCH) return TS_OK;
    const size_t row = 2 * (size_t)gram_tc_ld(S.m);
    for (int n = 0; n < S.N; ++n) {
      if (!S.fused[n]) continue;
      const int s = (int)X.dims[n], r = S.r[n];
      const int kk = S.solve == TS_SOLVE_RSVD ? S.kc[n] : 0;
      for (int t = t0; t < t0 + nt; ++t) {
        char* bt = static_cast<char*>(w.Bt[n]) + (size_t)t * w.bt_stride[n];
        if (kk)
          TS_TRY(pack_bf16(w.YOm + S.yom_off[n] + (size_t)t * kk, 1, (long)S.sweeps * kk, kk,
                           S.m, bt + (size_t)r * row, st));
        TS_TRY(pack_bf16(w.Y[n], 1, s, s, S.m, bt + (size_t)(r + kk) * row, st));
      }
    }
  }
  return TS_OK;
}

// Y_n Omega(sweep, n) for sweeps [t0, t0 + nt) of every mode, one product per mode.
template <typename T>
static ts_status rhs_times_omegas(const ts_tensor& X, const Shape& S, Work<T>& w, int t0, int nt,
                                  cudaStream_t st) {
  for (int n = 0; n < S.N; ++n) {
    const int k = S.kc[n];
    const long ld = (long)S.sweeps * k;
    const int s = (int)X.dims[n];
    if (s >= kTallMinS)
      TS_TRY(wide_nn<T>(S.m, nt * k, s, w.Y[n], s, w.Om + S.ob.off[n] + (size_t)t0 * k, ld,
                        w.YOm + S.yom_off[n] + (size_t)t0 * k, ld, 1, w.split.partial,
                        w.split.partial_elems, st));
    else
      TS_TRY(gemm<T>(S.m, nt * k, s, 1.0, mv<T>(w.Y[n], s, 1),
                     mv<T>(w.Om + S.ob.off[n] + (size_t)t0 * k, ld, 1), 0.0,
                     ov<T>(w.YOm + S.yom_off[n] + (size_t)t0 * k, ld, 1), &w.split, st));
  }
  return TS_OK;
}

static ts_status phase(const ts_options& opt, int i, cudaStream_t st) {
  if (opt.phase_events && opt.phase_events[i])
    TS_CUDA(cudaEventRecord((cudaEvent_t)opt.phase_events[i], st));
  return TS_OK;
}

template <typename T>
static ts_status als_impl(const ts_tensor& X, const Shape& S, const ts_options& opt, void* ws,
                          T* core, T* const* factors, double* residual_out, cudaStream_t st) {
  Work<T> w;
  Bump b{static_cast<char*>(ws)};
  carve<T>(X, S, residual_out != nullptr, b, w);
  const int N = S.N, m = S.m;
  TS_TRY(phase(opt, 0, st));
  TS_CUDA(cudaMemsetAsync(w.flag, 0, 256 + kGemmCounters * sizeof(unsigned), st));
  if (residual_out && X.format == TS_COO) TS_TRY(launch_fit_coo_norm(X, w.fitc, w.flag, st));
  auto fit = [&](double* out) -> ts_status {
    if (X.format == TS_COO)
      return launch_fit_coo<T>(X, S.ranks, core, (const T* const*)factors, w.fitc, out, st);
    return launch_fit_dense<T>(X, S.ranks, core, (const T* const*)factors, w.fitQ, w.fitacc, out,
                               st);
  };
  if (S.rrf) TS_TRY(rrf_all<T>(X, S, opt.seed, w, factors, st));
  TS_TRY(phase(opt, 1, st));
  if (S.solve == TS_SOLVE_RSVD) TS_TRY(launch_omegas<T>(opt.seed, S.ob, w.Om, st));
  if (S.kind == TS_TENSORSKETCH) {
    TS_TRY(launch_twiddles<T>(m, w.tw, st));
    TS_TRY(build_ts_tables<T>(X, S, opt.seed, 0, w, st));
    TS_TRY(phase(opt, 2, st));
    TS_TRY(sketch_rhs_all<T>(X, S, w, st));
    TS_TRY(phase(opt, 3, st));
    const int npass = opt.resketch_each_sweep ? 1 : S.sweeps;
    if (S.solve == TS_SOLVE_RSVD) TS_TRY(rhs_times_omegas<T>(X, S, w, 0, npass, st));
    TS_TRY(pack_rhs_bf16<T>(X, S, w, 0, npass, st));
  } else {
    TS_TRY(phase(opt, 2, st));
    if (S.coo_lev)
      for (int n = 0; n < N; ++n) TS_TRY(launch_fibre_index_build(X, w.fib[n], w.flag, st));
    TS_TRY(phase(opt, 3, st));
  }
  const T* chain[TS_MAX_ORDER];
  const int32_t* ctab[TS_MAX_ORDER];
  int64_t rows[TS_MAX_ORDER];
  int cols[TS_MAX_ORDER];
  for (int sweep = 0; sweep < S.sweeps; ++sweep) {
    if (S.kind == TS_TENSORSKETCH && opt.resketch_each_sweep && sweep > 0) {
      TS_TRY(build_ts_tables<T>(X, S, opt.seed, sweep, w, st));
      TS_TRY(sketch_rhs_all<T>(X, S, w, st));
      if (S.solve == TS_SOLVE_RSVD) TS_TRY(rhs_times_omegas<T>(X, S, w, sweep, 1, st));
      TS_TRY(pack_rhs_bf16<T>(X, S, w, sweep, 1, st));
    }
    for (int n = 0; n < N; ++n) {
      const T* Yn;
      if (S.kind == TS_TENSORSKETCH) {
        int nf = 0;
        for (int k = 0; k < N; ++k)
          if (k != n) {
            chain[nf] = factors[k];
            ctab[nf] = w.tab[n][k];
            rows[nf] = X.dims[k];
            cols[nf] = S.ranks[k];
            ++nf;
          }
        void* zb = (S.bf16gram && S.fused[n])
                       ? static_cast<char*>(w.Bt[n]) + (size_t)sweep * w.bt_stride[n]
                       : nullptr;
        TS_TRY(launch_ts_apply<T>(nf, chain, rows, cols, ctab, m, w.tw, w.spectra, w.ZW, st, zb,
                                  gram_tc_ld(m)));
        Yn = w.Y[n];
      } else {
        TS_TRY(launch_leverage<T>(X, n, S.ranks, (const T* const*)factors, m, opt.seed, sweep,
                                  w.ZW, w.Ylev, w.samples, w.levscr, st,
                                  S.kind == TS_LEVERAGE_DET, S.coo_lev ? &w.fib[n] : nullptr));
        Yn = w.Ylev;
      }
      CoreMap map{};
      map.order = N;
      map.n = n;
      for (int k = 0; k < N; ++k) map.ranks[k] = S.ranks[k];
      const long ldo = (long)S.sweeps * S.kc[n];
      const T* Om = w.Om ? w.Om + S.ob.off[n] + (size_t)sweep * S.kc[n] : nullptr;
      MatView<T> yv{};
      const MatView<T>* yom = nullptr;
      if (w.YOm) {
        yv = mv<T>(w.YOm + S.yom_off[n] + (size_t)sweep * S.kc[n], ldo, 1);
        yom = &yv;
      }
      Bf16Op bop{S.bf16gram ? static_cast<char*>(w.Bt[n]) + (size_t)sweep * w.bt_stride[n]
                            : nullptr,
                 S.kind == TS_TENSORSKETCH};
      const Bf16Op* bf = (S.bf16gram && S.fused[n]) ? &bop : nullptr;
      TS_TRY(solve_subproblem<T>(m, S.r[n], (int)X.dims[n], S.ranks[n], S.solve, S.kc[n],
                                 S.fp64solve, Om, ldo, yom, Yn, w, factors[n], core, map, st,
                                 bf));
    }
    if (residual_out && opt.track_fit) TS_TRY(fit(residual_out + sweep));
  }
  TS_TRY(phase(opt, 4, st));
  if (residual_out && !opt.track_fit) TS_TRY(fit(residual_out));
  TS_TRY(phase(opt, 5, st));
  return TS_OK;
}

// ---------------------------------------------------------------- graph replay

// Small per-device cache of instantiated CUDA graphs keyed by the full argument set.
// Capture runs on a library-owned stream (the legacy default stream cannot be
// captured); the executable graph is then launched on the caller's stream.
struct GraphEntry {
  std::string key;
  int device;
  cudaGraphExec_t exec;
};
static std::mutex g_graph_mu;
static std::vector<GraphEntry> g_graphs;  // most recent last
static cudaStream_t g_capture_stream[64] = {};
constexpr size_t kMaxGraphs = 8;

template <typename F>
static ts_status graph_replay(const std::string& key, F&& enqueue, cudaStream_t st) {
  int dev = 0;
  TS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return enqueue(st);
  std::lock_guard<std::mutex> lock(g_graph_mu);
  for (size_t i = 0; i < g_graphs.size(); ++i)
    if (g_graphs[i].device == dev && g_graphs[i].key == key) {
      GraphEntry e = g_graphs[i];
      g_graphs.erase(g_graphs.begin() + i);
      g_graphs.push_back(e);
      TS_CUDA(cudaGraphLaunch(e.exec, st));
      return TS_OK;
    }
  if (!g_capture_stream[dev])
    TS_CUDA(cudaStreamCreateWithFlags(&g_capture_stream[dev], cudaStreamNonBlocking));
  cudaStream_t cs = g_capture_stream[dev];
  TS_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  ts_status s = enqueue(cs);
  cudaGraph_t graph = nullptr;
  cudaError_t ec = cudaStreamEndCapture(cs, &graph);
  if (s != TS_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (ec != cudaSuccess)
    return fail(TS_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ec));
  cudaGraphExec_t exec = nullptr;
  ec = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ec != cudaSuccess)
    return fail(TS_ERR_CUDA, "graph instantiate failed: %s", cudaGetErrorString(ec));
  if (g_graphs.size() >= kMaxGraphs) {
    cudaGraphExecDestroy(g_graphs.front().exec);
    g_graphs.erase(g_graphs.begin());
  }
  g_graphs.push_back(GraphEntry{key, dev, exec});
  TS_CUDA(cudaGraphLaunch(exec, st));
  return TS_OK;
}

// ---------------------------------------------------------------- batched form

// Many independent dense tensors advanced together: every tensor keeps its own
// workspace region (the single-tensor layout), its setup (tables, one-pass sketches,
// Init-RRF, Gaussians, Y_n Omega) runs once in ts_batch_prepare, and each subproblem
// step of a sweep is one launch over the whole batch: the TensorSketch chains, the
// products [Z^T Z | Z^T Y Omega | Z^T Y], the single-block solves.  The per-tensor
// arguments of every launch live in device descriptor arrays written once by prepare,
// so the sweeps enqueue nothing but kernel launches (capturable in a CUDA graph).
struct BatchPlan {
  int count = 0, N = 0, sweeps = 0, dtype = TS_F32, solve = TS_SOLVE_RSVD;
  bool fp64 = false;
  int device = 0;
  std::vector<Shape> S;
  std::vector<ts_tensor> X;
  std::vector<void*> cores, factors;  // factors: count x N
  std::vector<int*> flags;
  std::vector<void*> fitQ, fitacc;
  void* chain = nullptr;  // TsChainJob<T> [N][count]
  void* gemm = nullptr;   // GemmJob<T> [sweeps][N][count]
  void* fused = nullptr;  // FusedArgs<T> [N][count]
  int spec_blocks[TS_MAX_ORDER] = {}, z_blocks[TS_MAX_ORDER] = {};
  int maxM[TS_MAX_ORDER] = {}, maxN[TS_MAX_ORDER] = {}, tile[TS_MAX_ORDER] = {};
  size_t chain_smem[TS_MAX_ORDER] = {}, fused_smem[TS_MAX_ORDER] = {};
  float tile_ms[TS_MAX_ORDER][2] = {};  // autotuner: product time per tile shape (32, 64)
};

static ts_status batch_check(int count, const ts_tensor* X, const int32_t* ranks,
                             const int32_t* m, int sweeps, const ts_options* opt) {
  if (count < 1 || !X || !ranks || !m || !opt)
    return fail(TS_ERR_INVALID_ARG, "ts_batch: need count >= 1 and non-NULL X, ranks, m, opt");
  if (opt->resketch_each_sweep || opt->gram_bf16 || opt->use_graph)
    return fail(TS_ERR_UNSUPPORTED,
                "ts_batch: resketch_each_sweep, gram_bf16 and use_graph are not offered");
  for (int i = 0; i < count; ++i) {
    if (X[i].format != TS_DENSE || X[i].order != X[0].order || X[i].dtype != X[0].dtype)
      return fail(TS_ERR_UNSUPPORTED, "ts_batch: tensor %d: dense tensors of one order and dtype",
                  i);
  }
  if (sweeps < 1) return fail(TS_ERR_SHAPE, "ts_batch: sweeps %d < 1", sweeps);
  return TS_OK;
}

static ts_status batch_shapes(int count, const ts_tensor* X, const int32_t* ranks,
                              const int32_t* m, int sweeps, const ts_options* opt,
                              std::vector<Shape>& S) {
  S.resize(count);
  const int N = X[0].order;
  for (int i = 0; i < count; ++i) {
    TS_TRY(plan_shape(&X[i], ranks + (size_t)i * N, TS_TENSORSKETCH, m[i], sweeps, opt, true,
                      S[i]));
    for (int n = 0; n < N; ++n)
      if (!S[i].fused[n])
        return fail(TS_ERR_UNSUPPORTED,
                    "ts_batch: tensor %d mode %d (r=%d, s=%lld) does not fit the single-block solve",
                    i, n, S[i].r[n], (long long)X[i].dims[n]);
  }
  return TS_OK;
}

template <typename T>
static size_t batch_desc_bytes(int count, int N, int sweeps) {
  Bump b;
  b.take<TsChainJob<T>>((size_t)N * count);
  b.take<GemmJob<T>>((size_t)sweeps * N * count);
  b.take<FusedArgs<T>>((size_t)N * count);
  return align_up(b.off, 256);
}

template <typename T>
static size_t batch_bytes(int count, const ts_tensor* X, const std::vector<Shape>& S) {
  const int N = X[0].order;
  size_t total = batch_desc_bytes<T>(count, N, S[0].sweeps);
  for (int i = 0; i < count; ++i) {
    Bump b;
    Work<T> w;
    carve<T>(X[i], S[i], true, b, w);
    total += align_up(b.off, 256);
  }
  return total;
}

// Setup of every tensor, then the descriptors of every (sweep, mode, tensor) and the
// autotuned product tiles.  Synchronises the stream.
template <typename T>
static ts_status batch_prepare_impl(BatchPlan& P, const ts_options& opt, char* ws,
                                    cudaStream_t st) {
  const int count = P.count, N = P.N, sweeps = P.sweeps;
  std::vector<Work<T>> W(count);
  size_t off = batch_desc_bytes<T>(count, N, sweeps);
  {
    Bump b{ws};
    P.chain = b.take<TsChainJob<T>>((size_t)N * count);
    P.gemm = b.take<GemmJob<T>>((size_t)sweeps * N * count);
    P.fused = b.take<FusedArgs<T>>((size_t)N * count);
  }
  for (int i = 0; i < count; ++i) {
    Bump b{ws + off};
    carve<T>(P.X[i], P.S[i], true, b, W[i]);
    off += align_up(b.off, 256);
  }
  // per-tensor setup, exactly as the single-tensor driver (seed of tensor i: seed + i)
  for (int i = 0; i < count; ++i) {
    const ts_tensor& X = P.X[i];
    const Shape& S = P.S[i];
    Work<T>& w = W[i];
    T* const* fac = reinterpret_cast<T* const*>(&P.factors[(size_t)i * N]);
    const uint64_t seed = opt.seed + (uint64_t)i;
    TS_CUDA(cudaMemsetAsync(w.flag, 0, 256 + kGemmCounters * sizeof(unsigned), st));
    if (S.rrf) TS_TRY(rrf_all<T>(X, S, seed, w, fac, st));
    if (S.solve == TS_SOLVE_RSVD) TS_TRY(launch_omegas<T>(seed, S.ob, w.Om, st));
    TS_TRY(launch_twiddles<T>(S.m, w.tw, st));
    TS_TRY(build_ts_tables<T>(X, S, seed, 0, w, st));
    TS_TRY(sketch_rhs_all<T>(X, S, w, st));
    if (S.solve == TS_SOLVE_RSVD) TS_TRY(rhs_times_omegas<T>(X, S, w, 0, S.sweeps, st));
    P.flags[i] = w.flag;
    P.fitQ[i] = w.fitQ;
    P.fitacc[i] = w.fitacc;
  }
  // descriptors
  std::vector<TsChainJob<T>> chain((size_t)N * count);
  std::vector<GemmJob<T>> gemm((size_t)sweeps * N * count);
  std::vector<FusedArgs<T>> fused((size_t)N * count);
  for (int n = 0; n < N; ++n) {
    P.spec_blocks[n] = P.z_blocks[n] = P.maxM[n] = P.maxN[n] = 0;
    P.chain_smem[n] = P.fused_smem[n] = 0;
    for (int i = 0; i < count; ++i) {
      const ts_tensor& X = P.X[i];
      const Shape& S = P.S[i];
      Work<T>& w = W[i];
      T* const* fac = reinterpret_cast<T* const*>(&P.factors[(size_t)i * N]);
      const T* cf[TS_MAX_ORDER];
      const int32_t* ct[TS_MAX_ORDER];
      int64_t rows[TS_MAX_ORDER];
      int cols[TS_MAX_ORDER];
      int nf = 0;
      for (int k = 0; k < N; ++k)
        if (k != n) {
          cf[nf] = fac[k];
          ct[nf] = w.tab[n][k];
          rows[nf] = X.dims[k];
          cols[nf] = S.ranks[k];
          ++nf;
        }
      TsChainJob<T>& cj = chain[(size_t)n * count + i];
      cj = make_chain_job<T>(nf, cf, rows, cols, ct, S.m, w.tw, w.spectra, w.ZW);
      P.spec_blocks[n] = std::max(P.spec_blocks[n], ceil_div(cj.d.total_cols, 2));
      P.z_blocks[n] = std::max(P.z_blocks[n], ceil_div(cj.ncols, 2));
      P.chain_smem[n] = std::max(P.chain_smem[n], chain_job_smem<T>(cj));
      const int r = S.r[n], k = S.kc[n], s = (int)X.dims[n], m = S.m;
      const bool rsvd = S.solve == TS_SOLVE_RSVD;
      const int kk = rsvd ? k : 0;
      const int Ncol = r + kk + s;
      const MatView<T> Zt = mv<T>(w.ZW, m, 1), Zm = mv<T>(w.ZW, 1, m);
      const MatView<T> Yv = mv<T>(w.Y[n], s, 1);
      for (int t = 0; t < sweeps; ++t) {
        GemmJob<T>& g = gemm[((size_t)t * N + n) * count + i];
        g.M = r;
        g.N = Ncol;
        g.K = m;
        g.A = Zt;
        g.B1 = Zm;
        g.n1 = r;
        if (rsvd) {
          g.B2 = mv<T>(w.YOm + S.yom_off[n] + (size_t)t * k, (long)S.sweeps * k, 1);
          g.n2 = r + k;
          g.B3 = Yv;
        } else {
          g.B2 = Yv;
          g.n2 = Ncol;
          g.B3 = Yv;
        }
        g.C = ov<T>(w.GW, Ncol, 1);
      }
      P.maxM[n] = std::max(P.maxM[n], r);
      P.maxN[n] = std::max(P.maxN[n], Ncol);
      CoreMap map{};
      map.order = N;
      map.n = n;
      for (int q = 0; q < N; ++q) map.ranks[q] = S.ranks[q];
      size_t sm = 0;
      TS_TRY(make_fused_args<T>(r, s, k, S.ranks[n], S.solve, S.fp64solve, w.GW, Ncol,
                                rsvd ? w.GW + r : nullptr, Ncol, w.GW + r + kk, Ncol, w.Mbuf,
                                w.CnT, fac[n], static_cast<T*>(P.cores[i]), map, w.flag,
                                &fused[(size_t)n * count + i], &sm));
      P.fused_smem[n] = std::max(P.fused_smem[n], sm);
    }
  }
  // longest work first within every launch (blocks start in index order, so the batch's
  // makespan is not set by a long solve that starts last)
  for (int n = 0; n < N; ++n) {
    std::vector<int> ord(count);
    std::vector<double> cost(count), ccost(count);
    for (int i = 0; i < count; ++i) {
      const Shape& S = P.S[i];
      const double r = S.r[n], k = S.kc[n], sn = (double)P.X[i].dims[n];
      cost[i] = r * (r + k) + 4.0 * k * sn;       // the single-block solve
      ccost[i] = (double)S.m * (r + 2.0 * S.Rmax);  // the FFT chain
      ord[i] = i;
    }
    auto sorted = [&](const std::vector<double>& c) {
      std::vector<int> o = ord;
      std::stable_sort(o.begin(), o.end(), [&](int a, int b) { return c[a] > c[b]; });
      return o;
    };
    const std::vector<int> of = sorted(cost), oc = sorted(ccost);
    std::vector<FusedArgs<T>> f2(count);
    std::vector<TsChainJob<T>> c2(count);
    for (int j = 0; j < count; ++j) {
      f2[j] = fused[(size_t)n * count + of[j]];
      c2[j] = chain[(size_t)n * count + oc[j]];
    }
    std::copy(f2.begin(), f2.end(), fused.begin() + (size_t)n * count);
    std::copy(c2.begin(), c2.end(), chain.begin() + (size_t)n * count);
    for (int t = 0; t < sweeps; ++t) {
      std::vector<GemmJob<T>> g2(count);
      for (int j = 0; j < count; ++j) g2[j] = gemm[((size_t)t * N + n) * count + of[j]];
      std::copy(g2.begin(), g2.end(), gemm.begin() + ((size_t)t * N + n) * count);
    }
  }
  TS_CUDA(cudaMemcpyAsync(P.chain, chain.data(), chain.size() * sizeof(chain[0]),
                          cudaMemcpyHostToDevice, st));
  TS_CUDA(cudaMemcpyAsync(P.gemm, gemm.data(), gemm.size() * sizeof(gemm[0]),
                          cudaMemcpyHostToDevice, st));
  TS_CUDA(cudaMemcpyAsync(P.fused, fused.data(), fused.size() * sizeof(fused[0]),
                          cudaMemcpyHostToDevice, st));
  // autotuner: time the batched product of every mode with both tile shapes, keep the
  // faster (the operands' values do not matter for the timing; the sweeps overwrite
  // the products)
  cudaEvent_t e0, e1;
  TS_CUDA(cudaEventCreate(&e0));
  TS_CUDA(cudaEventCreate(&e1));
  ts_status rc = TS_OK;
  for (int n = 0; n < N && rc == TS_OK; ++n) {
    const GemmJob<T>* jobs = static_cast<const GemmJob<T>*>(P.gemm) + (size_t)n * count;
    for (int v = 0; v < 2 && rc == TS_OK; ++v) {
      const int tile = v ? 64 : 32;
      rc = launch_gemm_batched<T>(jobs, count, P.maxM[n], P.maxN[n], tile, st);  // warm-up
      if (rc != TS_OK) break;
      cudaEventRecord(e0, st);
      for (int rep = 0; rep < 5 && rc == TS_OK; ++rep)
        rc = launch_gemm_batched<T>(jobs, count, P.maxM[n], P.maxN[n], tile, st);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        rc = fail(TS_ERR_CUDA, "ts_batch_prepare: autotuner timing failed");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      P.tile_ms[n][v] = ms / 5;
    }
    P.tile[n] = P.tile_ms[n][1] < P.tile_ms[n][0] ? 64 : 32;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  TS_TRY(rc);
  TS_CUDA(cudaStreamSynchronize(st));
  return TS_OK;
}

template <typename T>
static ts_status batch_sweeps_impl(const BatchPlan& P, int first, int nsweeps, cudaStream_t st) {
  const int count = P.count, N = P.N;
  const TsChainJob<T>* chain = static_cast<const TsChainJob<T>*>(P.chain);
  const GemmJob<T>* gemm = static_cast<const GemmJob<T>*>(P.gemm);
  const FusedArgs<T>* fused = static_cast<const FusedArgs<T>*>(P.fused);
  for (int t = first; t < first + nsweeps; ++t)
    for (int n = 0; n < N; ++n) {
      TS_TRY(launch_ts_apply_batched<T>(chain + (size_t)n * count, count, P.spec_blocks[n],
                                        P.z_blocks[n], P.chain_smem[n], st));
      TS_TRY(launch_gemm_batched<T>(gemm + ((size_t)t * N + n) * count, count, P.maxM[n],
                                    P.maxN[n], P.tile[n], st));
      TS_TRY(launch_lrls_fused_batched<T>(fused + (size_t)n * count, count, P.fp64,
                                          P.fused_smem[n], st));
    }
  return TS_OK;
}

}  // namespace ts

using namespace ts;

// ============================================================== C ABI

extern "C" ts_status tucker_als_workspace_bytes(const ts_tensor* X, const int32_t* ranks,
                                                int32_t kind, int32_t m, int32_t sweeps,
                                                const ts_options* opt, size_t* bytes_out) {
  clear_error();
  if (!bytes_out) return fail(TS_ERR_INVALID_ARG, "tucker_als_workspace_bytes: NULL bytes_out");
  Shape S;
  // Residual scratch is always counted (where a residual can be formed) so that one size
  // serves calls with and without residual_out; without it the carve only shrinks.
  TS_TRY(plan_shape(X, ranks, kind, m, sweeps, opt, X && X->format == TS_DENSE, S));
  const bool fit = X->format == TS_DENSE || (fit_coo_supported(*X) && fit_coo_model_ok(*X, ranks));
  Bump b;
  if (X->dtype == TS_F64) {
    Work<double> w;
    carve<double>(*X, S, fit, b, w);
  } else {
    Work<float> w;
    carve<float>(*X, S, fit, b, w);
  }
  *bytes_out = b.off;
  return TS_OK;
}

extern "C" ts_status tucker_als_sketched(const ts_tensor* X, const int32_t* ranks, int32_t kind,
                                         int32_t m, int32_t sweeps, const ts_options* opt,
                                         void* workspace, size_t workspace_bytes, void* core_out,
                                         void* const* factors_inout, double* residual_out,
                                         ts_stream stream) {
  clear_error();
  Shape S;
  TS_TRY(plan_shape(X, ranks, kind, m, sweeps, opt, residual_out != nullptr, S));
  if (!core_out || !factors_inout)
    return fail(TS_ERR_INVALID_ARG, "tucker_als_sketched: NULL core/factors");
  for (int k = 0; k < X->order; ++k)
    if (!factors_inout[k]) return fail(TS_ERR_INVALID_ARG, "tucker_als_sketched: factor %d NULL", k);
  size_t need = 0;
  TS_TRY(tucker_als_workspace_bytes(X, ranks, kind, m, sweeps, opt, &need));
  {
    // the carve of this very call (with or without the residual) must fit as well
    Bump b;
    if (X->dtype == TS_F64) {
      Work<double> w;
      carve<double>(*X, S, residual_out != nullptr, b, w);
    } else {
      Work<float> w;
      carve<float>(*X, S, residual_out != nullptr, b, w);
    }
    if (b.off > need) need = b.off;
  }
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255))
    return fail(TS_ERR_WORKSPACE, "tucker_als_sketched: need %zu bytes of 256-aligned workspace",
                need);
  cudaStream_t st = (cudaStream_t)stream;
  ts_options eo = *opt;
  if (opt->use_graph) eo.phase_events = nullptr;  // events inside a graph carry no timing
  auto enqueue = [&](cudaStream_t s) -> ts_status {
    if (X->dtype == TS_F64)
      return als_impl<double>(*X, S, eo, workspace, static_cast<double*>(core_out),
                              reinterpret_cast<double* const*>(factors_inout), residual_out, s);
    return als_impl<float>(*X, S, eo, workspace, static_cast<float*>(core_out),
                           reinterpret_cast<float* const*>(factors_inout), residual_out, s);
  };
  if (!opt->use_graph) return enqueue(st);
  // Key: every argument the enqueued work depends on (values and addresses).
  std::string key;
  auto put = [&](const void* p, size_t n) { key.append(static_cast<const char*>(p), n); };
  put(&X->order, sizeof(X->order));  // field by field: the struct has padding
  put(X->dims, sizeof(int64_t) * X->order);
  put(&X->format, sizeof(X->format));
  put(&X->dtype, sizeof(X->dtype));
  put(&X->values, sizeof(X->values));
  put(&X->indices, sizeof(X->indices));
  put(&X->nnz, sizeof(X->nnz));
  put(ranks, sizeof(int32_t) * X->order);
  put(&kind, sizeof(kind));
  put(&m, sizeof(m));
  put(&sweeps, sizeof(sweeps));
  put(&eo, sizeof(eo));
  put(&workspace, sizeof(workspace));
  put(&core_out, sizeof(core_out));
  put(factors_inout, sizeof(void*) * X->order);
  put(&residual_out, sizeof(residual_out));
  return graph_replay(key, enqueue, st);
}

extern "C" ts_status tensorsketch_input(const ts_tensor* X, int32_t mode,
                                        const int32_t* const* tables, int32_t m, void* Y_out,
                                        ts_stream stream) {
  clear_error();
  TS_TRY(check_tensor(X, "tensorsketch_input"));
  if (mode < 0 || mode >= X->order)
    return fail(TS_ERR_SHAPE, "tensorsketch_input: mode %d out of range", mode);
  if (!tables || !Y_out || m < 1)
    return fail(TS_ERR_INVALID_ARG, "tensorsketch_input: NULL tables/Y_out or m < 1");
  SketchJob job{};
  job.mode = mode;
  job.nbins = m;
  job.out = Y_out;
  for (int k = 0; k < X->order; ++k) {
    if (k != mode && !tables[k])
      return fail(TS_ERR_INVALID_ARG, "tensorsketch_input: table %d is NULL", k);
    job.tables[k] = k == mode ? nullptr : tables[k];
  }
  cudaStream_t st = (cudaStream_t)stream;
  return X->dtype == TS_F64 ? launch_input_sketch<double>(*X, &job, 1, nullptr, st)
                            : launch_input_sketch<float>(*X, &job, 1, nullptr, st);
}

// ---------------------------------------------------------------- Init-RRF, one mode

static ts_status rrf_check(const ts_tensor* X, int32_t mode, int32_t R, int32_t k1, int32_t k2) {
  TS_TRY(check_tensor(X, "range_finder_init"));
  if (mode < 0 || mode >= X->order) return fail(TS_ERR_SHAPE, "range_finder_init: bad mode");
  const int64_t K = prod_other(X->dims, X->order, mode);
  if (!(R >= 1 && R <= k1 && k1 <= k2 && k1 <= X->dims[mode] && k2 <= K && k1 <= kMaxEig))
    return fail(TS_ERR_SHAPE,
                "range_finder_init: need 1 <= R <= k1 <= min(k2, dims[mode]), k2 <= %lld, k1 <= %d",
                (long long)K, kMaxEig);
  return TS_OK;
}

template <typename T>
struct RrfWork {
  int* flag;
  unsigned* counters;
  int32_t* tabs[TS_MAX_ORDER];
  T *Wt, *Gm, *Bm, *K, *Fm;
  GemmSplit<T> split;
};

template <typename T>
static size_t rrf_carve(const ts_tensor& X, int mode, int R, int k1, int k2, Bump& b,
                        RrfWork<T>& w) {
  memset(&w, 0, sizeof(w));
  w.flag = b.take<int>(64);
  w.counters = b.take<unsigned>(kGemmCounters);
  for (int k = 0; k < X.order; ++k) w.tabs[k] = k == mode ? nullptr : b.take<int32_t>(X.dims[k]);
  const int64_t s = X.dims[mode];
  w.Wt = b.take<T>((size_t)k2 * s);
  w.Gm = b.take<T>((size_t)k2 * k1);
  w.Bm = b.take<T>((size_t)s * k1);
  w.K = b.take<T>((size_t)k1 * k1);
  w.Fm = b.take<T>((size_t)k1 * R);
  const size_t pm = (size_t)s * k1 > (size_t)k1 * k1 ? (size_t)s * k1 : (size_t)k1 * k1;
  w.split.partial_elems = 32 * pm;
  w.split.partial = b.take<T>(w.split.partial_elems);
  w.split.counters = w.counters;
  w.split.ncounters = kGemmCounters;
  return b.off;
}

extern "C" size_t range_finder_init_scratch_bytes(const ts_tensor* X, int32_t mode, int32_t R,
                                                  int32_t k1, int32_t k2) {
  if (rrf_check(X, mode, R, k1, k2) != TS_OK) return 0;
  Bump b;
  if (X->dtype == TS_F64) {
    RrfWork<double> w;
    return rrf_carve<double>(*X, mode, R, k1, k2, b, w);
  }
  RrfWork<float> w;
  return rrf_carve<float>(*X, mode, R, k1, k2, b, w);
}

template <typename T>
static ts_status rrf_one(const ts_tensor& X, int mode, int R, int k1, int k2, uint64_t seed,
                         T* A_out, void* scratch, cudaStream_t st) {
  Bump b{static_cast<char*>(scratch)};
  RrfWork<T> w;
  rrf_carve<T>(X, mode, R, k1, k2, b, w);
  TS_CUDA(cudaMemsetAsync(w.flag, 0, 256 + kGemmCounters * sizeof(unsigned), st));
  SketchJob job{};
  job.mode = mode;
  job.nbins = k2;
  job.out = w.Wt;
  for (int k = 0; k < X.order; ++k) {
    if (k != mode)
      TS_TRY(launch_hash_table(seed, TS_PURPOSE_RRF_HASH, 0, mode, k, X.dims[k], k2, w.tabs[k], st));
    job.tables[k] = w.tabs[k];
  }
  TS_TRY(launch_input_sketch<T>(X, &job, 1, w.flag, st));
  const int s = (int)X.dims[mode];
  TS_TRY(launch_gaussian<T>(seed, make_tag(TS_PURPOSE_RRF_GAUSS, 0, mode, 0), (int64_t)k2 * k1,
                            1.0 / sqrt((double)k1), w.Gm, st));
  TS_TRY(gemm<T>(s, k1, k2, 1.0, mv<T>(w.Wt, 1, s), mv<T>(w.Gm, k1, 1), 0.0, ov<T>(w.Bm, k1, 1),
                 &w.split, st));
  TS_TRY(gemm<T>(k1, k1, s, 1.0, mv<T>(w.Bm, 1, k1), mv<T>(w.Bm, k1, 1), 0.0, ov<T>(w.K, k1, 1),
                 &w.split, st));
  TS_TRY(launch_eig_small<T>(k1, R, w.K, nullptr, k1, nullptr, w.Fm, nullptr, false, w.flag, st));
  CoreMap none{};
  return launch_finalize<T>(s, R, w.Bm, k1, 1, k1, w.Fm, A_out, nullptr, 0, nullptr, none, st,
                            w.split.partial, w.split.partial_elems * sizeof(T));
}

extern "C" ts_status range_finder_init(const ts_tensor* X, int32_t mode, int32_t R, int32_t k1,
                                       int32_t k2, uint64_t seed, void* A_out, void* scratch,
                                       size_t scratch_bytes, ts_stream stream) {
  clear_error();
  TS_TRY(rrf_check(X, mode, R, k1, k2));
  if (!A_out) return fail(TS_ERR_INVALID_ARG, "range_finder_init: A_out is NULL");
  const size_t need = range_finder_init_scratch_bytes(X, mode, R, k1, k2);
  if (!scratch || scratch_bytes < need || ((uintptr_t)scratch & 255))
    return fail(TS_ERR_WORKSPACE, "range_finder_init: need %zu bytes of 256-aligned scratch", need);
  cudaStream_t st = (cudaStream_t)stream;
  return X->dtype == TS_F64
             ? rrf_one<double>(*X, mode, R, k1, k2, seed, static_cast<double*>(A_out), scratch, st)
             : rrf_one<float>(*X, mode, R, k1, k2, seed, static_cast<float*>(A_out), scratch, st);
}

// ---------------------------------------------------------------- one subproblem

static ts_status lrls_check(int32_t m, int32_t r, int32_t s, int32_t R, int32_t dtype,
                            int32_t solve, int32_t oversample, int32_t fp64, int* kc) {
  if (dtype != TS_F32 && dtype != TS_F64) return fail(TS_ERR_INVALID_ARG, "ts_lrls: bad dtype");
  if (solve != TS_SOLVE_RSVD && solve != TS_SOLVE_EXACT)
    return fail(TS_ERR_INVALID_ARG, "ts_lrls: bad solve kind");
  if (m < 1 || r < 1 || s < 1 || R < 1 || R > r || R > s || r > m)
    return fail(TS_ERR_SHAPE, "ts_lrls: need 1 <= R <= min(r, s) and r <= m");
  *kc = rsvd_width(R, oversample < 0 ? 5 : oversample, r, s);
  const bool q64 = fp64 && dtype == TS_F32;
  const size_t tsz = dtype_size(dtype);
  if (fused_ok(r, s, *kc, R, solve, tsz, q64)) return TS_OK;
  if (solve == TS_SOLVE_RSVD) {
    if (*kc > kMaxEig) return fail(TS_ERR_SHAPE, "ts_lrls: RSVD width k=%d > %d", *kc, kMaxEig);
    if (rsvd_stage1_smem_bytes(r, *kc, tsz, q64) > kMaxSmem &&
        qr_only_smem_bytes(r, *kc, q64, tsz) > kMaxSmem)
      return fail(TS_ERR_SHAPE, "ts_lrls: r=%d, k=%d too large for the RSVD solve", r, *kc);
    return TS_OK;
  }
  if (solve == TS_SOLVE_EXACT && (r > kMaxEig || chol_solve_smem_bytes(r, dtype_size(dtype)) > kMaxSmem))
    return fail(TS_ERR_SHAPE, "ts_lrls: exact limit r <= %d", kMaxEig);
  return TS_OK;
}

template <typename T>
static size_t lrls_carve(int m, int r, int s, int R, int solve, int kc, bool fp64, Bump& b,
                         Work<T>& w) {
  memset(&w, 0, sizeof(w));
  w.flag = b.take<int>(64);
  w.counters = b.take<unsigned>(kGemmCounters);
  const int k = kc;
  const int eign = solve == TS_SOLVE_EXACT ? (r > k ? r : k) : k;
  const bool fused = fused_ok(r, s, kc, R, solve, sizeof(T), fp64);
  w.ZW = b.take<T>((size_t)m * (r + k));
  w.GW = b.take<T>((size_t)r * (r + k + (fused ? s : 0)));
  if (!fused && solve == TS_SOLVE_RSVD && rsvd_stage1_smem_bytes(r, k, sizeof(T), fp64) > kMaxSmem) {
    w.Ginv = b.take<T>((size_t)r * r);
    w.NS1 = b.take<T>(2 * (size_t)r * r);
    w.NS2 = b.take<T>((size_t)r * r);
    w.Cb = b.take<T>((size_t)r * k);
  }
  w.Mbuf = fused ? b.take<T>((size_t)(solve == TS_SOLVE_RSVD ? k : r) * s) : nullptr;
  w.Om = b.take<T>((size_t)s * k);
  w.Q = b.take<T>((size_t)r * k);
  w.E = b.take<T>((size_t)r * k);
  w.Mm = b.take<T>((size_t)m * k);
  w.D = b.take<T>((size_t)k * s);
  w.K = b.take<T>((size_t)eign * eign);
  w.Fm = b.take<T>((size_t)eign * R);
  if (solve == TS_SOLVE_EXACT) {
    w.H = b.take<T>((size_t)r * s);
    w.Xs = b.take<T>((size_t)r * s);
  }
  size_t pm = (size_t)r * (r + k);
  const size_t cands[] = {(size_t)m * k, (size_t)k * s, (size_t)eign * eign,
                          solve == TS_SOLVE_EXACT ? (size_t)r * s : 0};
  for (size_t c : cands)
    if (c > pm) pm = c;
  w.split.partial_elems = 32 * pm;
  w.split.partial = b.take<T>(w.split.partial_elems);
  w.split.counters = w.counters;
  w.split.ncounters = kGemmCounters;
  return b.off;
}

extern "C" size_t ts_lrls_scratch_bytes(int32_t m, int32_t r, int32_t s, int32_t R, int32_t solve,
                                        int32_t oversample, int32_t dtype) {
  size_t best = 0;
  for (int f64 = 0; f64 < 2; ++f64) {  // enough for either supported precision of the solve
    int kc;
    if (lrls_check(m, r, s, R, dtype, solve, oversample, f64, &kc) != TS_OK) continue;
    Bump b;
    if (dtype == TS_F64) {
      Work<double> w;
      lrls_carve<double>(m, r, s, R, solve, kc, false, b, w);
    } else {
      Work<float> w;
      lrls_carve<float>(m, r, s, R, solve, kc, f64 != 0, b, w);
    }
    if (b.off > best) best = b.off;
  }
  if (best) clear_error();
  return best;
}

template <typename T>
static ts_status lrls_one(int m, int r, int s, int R, int solve, int kc, bool fp64, const void* Z,
                          const void* Y, uint64_t seed, int sweep, int n, void* CnT_out,
                          void* A_out, void* scratch, cudaStream_t st) {
  Bump b{static_cast<char*>(scratch)};
  Work<T> w;
  lrls_carve<T>(m, r, s, R, solve, kc, fp64, b, w);
  w.CnT = static_cast<T*>(CnT_out);
  TS_CUDA(cudaMemsetAsync(w.flag, 0, 256 + kGemmCounters * sizeof(unsigned), st));
  TS_CUDA(cudaMemcpyAsync(w.ZW, Z, sizeof(T) * (size_t)m * r, cudaMemcpyDeviceToDevice, st));
  if (solve == TS_SOLVE_RSVD)
    TS_TRY(launch_gaussian<T>(seed, make_tag(TS_PURPOSE_RSVD_GAUSS, sweep, n, 0), (int64_t)s * kc,
                              1.0, w.Om, st));
  CoreMap none{};
  return solve_subproblem<T>(m, r, s, R, solve, kc, fp64, w.Om, kc, nullptr,
                             static_cast<const T*>(Y), w,
                             static_cast<T*>(A_out), nullptr, none, st);
}

extern "C" ts_status ts_lrls_solve(int32_t m, int32_t r, int32_t s, int32_t R, int32_t dtype,
                                   const void* Z_colmajor, const void* Y, int32_t solve,
                                   uint64_t seed, int32_t sweep, int32_t n, int32_t oversample,
                                   int32_t solve_fp64, void* CnT_out, void* A_out, void* scratch,
                                   size_t scratch_bytes, ts_stream stream) {
  clear_error();
  int kc;
  TS_TRY(lrls_check(m, r, s, R, dtype, solve, oversample, solve_fp64, &kc));
  if (!Z_colmajor || !Y || !CnT_out || !A_out)
    return fail(TS_ERR_INVALID_ARG, "ts_lrls_solve: NULL argument");
  if (sweep < 0 || sweep >= (1 << 24) || n < 0 || n > 255)
    return fail(TS_ERR_INVALID_ARG, "ts_lrls_solve: sweep/n out of range");
  const size_t need = ts_lrls_scratch_bytes(m, r, s, R, solve, oversample, dtype);
  if (!scratch || scratch_bytes < need || ((uintptr_t)scratch & 255))
    return fail(TS_ERR_WORKSPACE, "ts_lrls_solve: need %zu bytes of 256-aligned scratch", need);
  cudaStream_t st = (cudaStream_t)stream;
  const bool fp64 = solve_fp64 != 0 && dtype == TS_F32;
  return dtype == TS_F64 ? lrls_one<double>(m, r, s, R, solve, kc, false, Z_colmajor, Y, seed,
                                            sweep, n, CnT_out, A_out, scratch, st)
                         : lrls_one<float>(m, r, s, R, solve, kc, fp64, Z_colmajor, Y, seed,
                                           sweep, n, CnT_out, A_out, scratch, st);
}

// ---------------------------------------------------------------- leverage sketch

// Scratch of the standalone leverage sketches: [flag ints | samples | scores, cdf,
// probabilities (+ the deterministic selection's scores) | COO: the mode's fibre index].
static size_t lev_carve(const ts_tensor& X, int mode, int m, Bump& b, int** flag, int32_t** smp,
                        double** lv, FibreIndex* F) {
  *flag = b.take<int>(64);
  *smp = b.take<int32_t>((size_t)m * (X.order - 1));
  *lv = b.take<double>(leverage_scratch_doubles(X, mode, m));
  if (X.format == TS_COO) *F = fibre_index_carve(X, mode, b);
  return b.off;
}

static ts_status lev_check(const ts_tensor* X, int32_t mode, const int32_t* ranks,
                           const void* const* factors, int32_t m, const void* Z_out,
                           const void* Y_out, const char* who) {
  TS_TRY(check_tensor(X, who));
  if (mode < 0 || mode >= X->order || m < 1) return fail(TS_ERR_SHAPE, "%s: bad mode or m", who);
  if (!ranks || !factors || !Z_out || !Y_out) return fail(TS_ERR_INVALID_ARG, "%s: NULL argument", who);
  for (int k = 0; k < X->order; ++k)
    if (k != mode && (!factors[k] || ranks[k] < 1))
      return fail(TS_ERR_INVALID_ARG, "%s: bad factor %d", who, k);
  if (X->format == TS_COO) {
    if (X->nnz >= (int64_t(1) << 30))
      return fail(TS_ERR_UNSUPPORTED, "%s: COO tensors take < 2^30 nonzeros", who);
    if (!fibre_keys_fit(*X, mode))
      return fail(TS_ERR_UNSUPPORTED, "%s: fibre keys of mode %d exceed 64 bits", who, mode);
  }
  return TS_OK;
}

extern "C" size_t ts_leverage_sketch_scratch_bytes(const ts_tensor* X, int32_t mode, int32_t m) {
  if (check_tensor(X, "ts_leverage_sketch") != TS_OK || mode < 0 || mode >= X->order || m < 1)
    return 0;
  Bump b;
  int* f;
  int32_t* smp;
  double* lv;
  FibreIndex F;
  return lev_carve(*X, mode, m, b, &f, &smp, &lv, &F);
}

static ts_status lev_run(const ts_tensor* X, int32_t mode, const int32_t* ranks,
                         const void* const* factors, int32_t m, uint64_t seed, int32_t sweep,
                         void* Z_out, void* Y_out, int32_t* samples_out, void* scratch,
                         size_t scratch_bytes, ts_stream stream, bool det, const char* who) {
  const size_t need = ts_leverage_sketch_scratch_bytes(X, mode, m);
  if (!scratch || scratch_bytes < need || ((uintptr_t)scratch & 255))
    return fail(TS_ERR_WORKSPACE, "%s: need %zu bytes of 256-aligned scratch", who, need);
  Bump b{static_cast<char*>(scratch)};
  int* flag;
  int32_t* smp;
  double* lv;
  FibreIndex F{};
  lev_carve(*X, mode, m, b, &flag, &smp, &lv, &F);
  if (samples_out) smp = samples_out;
  cudaStream_t st = (cudaStream_t)stream;
  TS_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
  const FibreIndex* fib = nullptr;
  if (X->format == TS_COO) {
    TS_TRY(launch_fibre_index_build(*X, F, flag, st));
    fib = &F;
  }
  if (X->dtype == TS_F64)
    return launch_leverage<double>(*X, mode, ranks, reinterpret_cast<const double* const*>(factors),
                                   m, seed, sweep, static_cast<double*>(Z_out),
                                   static_cast<double*>(Y_out), smp, lv, st, det, fib);
  return launch_leverage<float>(*X, mode, ranks, reinterpret_cast<const float* const*>(factors), m,
                                seed, sweep, static_cast<float*>(Z_out),
                                static_cast<float*>(Y_out), smp, lv, st, det, fib);
}

extern "C" ts_status ts_leverage_sketch(const ts_tensor* X, int32_t mode, const int32_t* ranks,
                                        const void* const* factors, int32_t m, uint64_t seed,
                                        int32_t sweep, void* Z_out, void* Y_out,
                                        int32_t* samples_out, void* scratch, size_t scratch_bytes,
                                        ts_stream stream) {
  clear_error();
  TS_TRY(lev_check(X, mode, ranks, factors, m, Z_out, Y_out, "ts_leverage_sketch"));
  if (sweep < 0 || sweep >= (1 << 24))
    return fail(TS_ERR_INVALID_ARG, "ts_leverage_sketch: sweep out of range");
  return lev_run(X, mode, ranks, factors, m, seed, sweep, Z_out, Y_out, samples_out, scratch,
                 scratch_bytes, stream, false, "ts_leverage_sketch");
}

extern "C" ts_status ts_leverage_sketch_det(const ts_tensor* X, int32_t mode, const int32_t* ranks,
                                            const void* const* factors, int32_t m, void* Z_out,
                                            void* Y_out, int32_t* samples_out, void* scratch,
                                            size_t scratch_bytes, ts_stream stream) {
  clear_error();
  TS_TRY(lev_check(X, mode, ranks, factors, m, Z_out, Y_out, "ts_leverage_sketch_det"));
  return lev_run(X, mode, ranks, factors, m, 0, 0, Z_out, Y_out, samples_out, scratch,
                 scratch_bytes, stream, true, "ts_leverage_sketch_det");
}

// ---------------------------------------------------------------- fitness

extern "C" size_t ts_fitness_scratch_bytes(const ts_tensor* X, const int32_t* ranks) {
  if (check_tensor(X, "ts_fitness") != TS_OK || !ranks) return 0;
  Bump b;
  if (X->format == TS_COO) {
    b.take<int>(64);
    fit_coo_carve(*X, ranks, b);
    return b.off;
  }
  if (X->dtype == TS_F64)
    b.take<double>(fit_dense_scratch_elems<double>(*X, ranks));
  else
    b.take<float>(fit_dense_scratch_elems<float>(*X, ranks));
  b.take<double>(2);
  return b.off;
}

extern "C" ts_status ts_fitness(const ts_tensor* X, const int32_t* ranks, const void* core,
                                const void* const* factors, double* residual_out, void* scratch,
                                size_t scratch_bytes, ts_stream stream) {
  clear_error();
  TS_TRY(check_tensor(X, "ts_fitness"));
  if (!ranks || !core || !factors || !residual_out)
    return fail(TS_ERR_INVALID_ARG, "ts_fitness: NULL argument");
  if (X->format == TS_COO && (!fit_coo_supported(*X) || !fit_coo_model_ok(*X, ranks)))
    return fail(TS_ERR_UNSUPPORTED,
                "ts_fitness: COO residual needs < 2^30 nonzeros, fibre keys of the largest mode "
                "within 64 bits, a core <= 200 KB and a last rank <= 64");
  for (int k = 0; k < X->order; ++k)
    if (!factors[k] || ranks[k] < 1) return fail(TS_ERR_INVALID_ARG, "ts_fitness: bad factor %d", k);
  const size_t need = ts_fitness_scratch_bytes(X, ranks);
  if (!scratch || scratch_bytes < need || ((uintptr_t)scratch & 255))
    return fail(TS_ERR_WORKSPACE, "ts_fitness: need %zu bytes of 256-aligned scratch", need);
  Bump b{static_cast<char*>(scratch)};
  cudaStream_t st = (cudaStream_t)stream;
  if (X->format == TS_COO) {
    int* flag = b.take<int>(64);
    const FitCooWork w = fit_coo_carve(*X, ranks, b);
    TS_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
    TS_TRY(launch_fit_coo_norm(*X, w, flag, st));
    if (X->dtype == TS_F64)
      return launch_fit_coo<double>(*X, ranks, static_cast<const double*>(core),
                                    reinterpret_cast<const double* const*>(factors), w,
                                    residual_out, st);
    return launch_fit_coo<float>(*X, ranks, static_cast<const float*>(core),
                                 reinterpret_cast<const float* const*>(factors), w, residual_out,
                                 st);
  }
  if (X->dtype == TS_F64) {
    double* q = b.take<double>(fit_dense_scratch_elems<double>(*X, ranks));
    double* acc = b.take<double>(2);
    return launch_fit_dense<double>(*X, ranks, static_cast<const double*>(core),
                                    reinterpret_cast<const double* const*>(factors), q, acc,
                                    residual_out, st);
  }
  float* q = b.take<float>(fit_dense_scratch_elems<float>(*X, ranks));
  double* acc = b.take<double>(2);
  return launch_fit_dense<float>(*X, ranks, static_cast<const float*>(core),
                                 reinterpret_cast<const float* const*>(factors), q, acc,
                                 residual_out, st);
}

// ---------------------------------------------------------------- CP-Sketch-Tucker (Alg. 6)

namespace ts {

static ts_status cp_check(const ts_tensor* X, int R_cp, const int32_t* tranks, int m, int sweeps,
                          const ts_options* opt, bool want_residual, Shape& S) {
  TS_TRY(plan_shape(X, tranks, TS_TENSORSKETCH, m, sweeps, opt, false, S));
  if (want_residual && X->format == TS_COO) {
    int rk[TS_MAX_ORDER];
    for (int k = 0; k < X->order; ++k) rk[k] = R_cp;
    if (!fit_coo_supported(*X) || !fit_coo_model_ok(*X, rk))
      return fail(TS_ERR_UNSUPPORTED, "cp_via_tucker: COO residual outside its limits");
  }
  long core = 1;
  int rmin = 1 << 30;
  for (int k = 0; k < X->order; ++k) {
    core *= tranks[k];
    if (tranks[k] < rmin) rmin = tranks[k];
  }
  if (R_cp < 1 || R_cp > rmin || R_cp > kMaxEig || core > 65536 ||
      chol_solve_smem_bytes(R_cp, dtype_size(X->dtype)) > kMaxSmem)
    return fail(TS_ERR_SHAPE, "cp_via_tucker: need 1 <= R_cp <= min(tucker_ranks), R_cp <= %d and "
                              "prod(tucker_ranks) <= 65536", kMaxEig);
  return TS_OK;
}

// Alg. 6 layout: the Tucker workspace first, then the core, B^(n), A^(n), CP scratch
// and the residual buffers.
template <typename T>
struct CpWork {
  T* core;
  T* B[TS_MAX_ORDER];
  T* A[TS_MAX_ORDER];
  T* cps;
  T* D;
  T* fq;
  double* acc;
  FitCooWork fitc;  // COO residual
};

template <typename T>
static size_t cp_carve(const ts_tensor& X, const Shape& S, int Rc, Bump& b, CpWork<T>& c) {
  Work<T> w;
  carve<T>(X, S, false, b, w);
  long core = 1, dcore = 1;
  int rk[TS_MAX_ORDER];
  for (int k = 0; k < S.N; ++k) {
    core *= S.ranks[k];
    dcore *= Rc;
    rk[k] = Rc;
  }
  c.core = b.take<T>((size_t)core);
  for (int k = 0; k < S.N; ++k) c.B[k] = b.take<T>((size_t)X.dims[k] * S.ranks[k]);
  for (int k = 0; k < S.N; ++k) c.A[k] = b.take<T>((size_t)S.ranks[k] * Rc);
  c.cps = b.take<T>(cp_core_scratch_elems<T>(S.N, S.ranks, Rc));
  c.D = b.take<T>((size_t)dcore);
  c.fq = X.format == TS_DENSE ? b.take<T>(fit_dense_scratch_elems<T>(X, rk)) : nullptr;
  c.acc = b.take<double>(2);
  if (X.format == TS_COO) c.fitc = fit_coo_carve(X, rk, b);
  return b.off;
}

template <typename T>
static ts_status cp_impl(const ts_tensor& X, const Shape& S, const ts_options& opt, int Rc,
                         int cp_sweeps, void* ws, T* const* out, double* residual_out,
                         cudaStream_t st) {
  Bump b{static_cast<char*>(ws)};
  CpWork<T> c;
  cp_carve<T>(X, S, Rc, b, c);
  ts_options o = opt;
  o.track_fit = 0;
  o.init_given = 0;
  TS_TRY(als_impl<T>(X, S, o, ws, c.core, c.B, nullptr, st));
  int* flag = static_cast<int*>(ws);  // the Tucker workspace's breakdown flag
  TS_TRY(cp_als_core<T>(S.N, S.ranks, Rc, cp_sweeps, c.core, c.A, c.cps, flag, st));
  for (int k = 0; k < S.N; ++k)
    TS_TRY(gemm<T>((int)X.dims[k], Rc, S.ranks[k], 1.0, mv<T>(c.B[k], S.ranks[k], 1),
                   mv<T>(c.A[k], Rc, 1), 0.0, ov<T>(out[k], Rc, 1), nullptr, st));
  if (residual_out) {
    int rk[TS_MAX_ORDER];
    for (int k = 0; k < S.N; ++k) rk[k] = Rc;
    TS_TRY(launch_superdiag<T>(S.N, Rc, c.D, st));
    if (X.format == TS_COO) {
      TS_TRY(launch_fit_coo_norm(X, c.fitc, flag, st));
      TS_TRY(launch_fit_coo<T>(X, rk, c.D, (const T* const*)out, c.fitc, residual_out, st));
    } else {
      TS_TRY(launch_fit_dense<T>(X, rk, c.D, (const T* const*)out, c.fq, c.acc, residual_out,
                                 st));
    }
  }
  return TS_OK;
}

}  // namespace ts

extern "C" ts_status cp_via_tucker_workspace_bytes(const ts_tensor* X, int32_t R_cp,
                                                   const int32_t* tucker_ranks, int32_t m,
                                                   int32_t tucker_sweeps, const ts_options* opt,
                                                   size_t* bytes_out) {
  clear_error();
  if (!bytes_out) return fail(TS_ERR_INVALID_ARG, "cp_via_tucker_workspace_bytes: NULL bytes_out");
  Shape S;
  TS_TRY(cp_check(X, R_cp, tucker_ranks, m, tucker_sweeps, opt, false, S));
  Bump b;
  if (X->dtype == TS_F64) {
    CpWork<double> c;
    *bytes_out = cp_carve<double>(*X, S, R_cp, b, c);
  } else {
    CpWork<float> c;
    *bytes_out = cp_carve<float>(*X, S, R_cp, b, c);
  }
  return TS_OK;
}

extern "C" ts_status cp_via_tucker(const ts_tensor* X, int32_t R_cp, const int32_t* tucker_ranks,
                                   int32_t m, int32_t tucker_sweeps, int32_t cp_sweeps,
                                   const ts_options* opt, void* workspace, size_t workspace_bytes,
                                   void* const* cp_factors_out, double* residual_out,
                                   ts_stream stream) {
  clear_error();
  Shape S;
  TS_TRY(cp_check(X, R_cp, tucker_ranks, m, tucker_sweeps, opt, residual_out != nullptr, S));
  if (cp_sweeps < 0) return fail(TS_ERR_SHAPE, "cp_via_tucker: cp_sweeps < 0");
  if (!cp_factors_out) return fail(TS_ERR_INVALID_ARG, "cp_via_tucker: NULL cp_factors_out");
  for (int k = 0; k < X->order; ++k)
    if (!cp_factors_out[k]) return fail(TS_ERR_INVALID_ARG, "cp_via_tucker: factor %d NULL", k);
  size_t need = 0;
  TS_TRY(cp_via_tucker_workspace_bytes(X, R_cp, tucker_ranks, m, tucker_sweeps, opt, &need));
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255))
    return fail(TS_ERR_WORKSPACE, "cp_via_tucker: need %zu bytes of 256-aligned workspace", need);
  cudaStream_t st = (cudaStream_t)stream;
  if (X->dtype == TS_F64)
    return cp_impl<double>(*X, S, *opt, R_cp, cp_sweeps, workspace,
                           reinterpret_cast<double* const*>(cp_factors_out), residual_out, st);
  return cp_impl<float>(*X, S, *opt, R_cp, cp_sweeps, workspace,
                        reinterpret_cast<float* const*>(cp_factors_out), residual_out, st);
}

// ---------------------------------------------------------------- batched form

extern "C" ts_status ts_batch_workspace_bytes(int32_t count, const ts_tensor* X,
                                              const int32_t* ranks, const int32_t* m,
                                              int32_t sweeps, const ts_options* opt,
                                              size_t* bytes_out) {
  clear_error();
  if (!bytes_out) return fail(TS_ERR_INVALID_ARG, "ts_batch_workspace_bytes: NULL bytes_out");
  TS_TRY(batch_check(count, X, ranks, m, sweeps, opt));
  std::vector<Shape> S;
  TS_TRY(batch_shapes(count, X, ranks, m, sweeps, opt, S));
  *bytes_out = X[0].dtype == TS_F64 ? batch_bytes<double>(count, X, S)
                                    : batch_bytes<float>(count, X, S);
  return TS_OK;
}

extern "C" ts_status ts_batch_prepare(int32_t count, const ts_tensor* X, const int32_t* ranks,
                                      const int32_t* m, int32_t sweeps, const ts_options* opt,
                                      void* workspace, size_t workspace_bytes,
                                      void* const* cores, void* const* factors,
                                      ts_batch* batch_out, ts_stream stream) {
  clear_error();
  if (!batch_out) return fail(TS_ERR_INVALID_ARG, "ts_batch_prepare: NULL batch_out");
  *batch_out = nullptr;
  TS_TRY(batch_check(count, X, ranks, m, sweeps, opt));
  if (!cores || !factors) return fail(TS_ERR_INVALID_ARG, "ts_batch_prepare: NULL cores/factors");
  const int N = X[0].order;
  for (int i = 0; i < count; ++i) {
    if (!cores[i]) return fail(TS_ERR_INVALID_ARG, "ts_batch_prepare: core %d NULL", i);
    for (int k = 0; k < N; ++k)
      if (!factors[(size_t)i * N + k])
        return fail(TS_ERR_INVALID_ARG, "ts_batch_prepare: factor %d of tensor %d NULL", k, i);
  }
  std::unique_ptr<BatchPlan> P(new BatchPlan);
  TS_TRY(batch_shapes(count, X, ranks, m, sweeps, opt, P->S));
  const size_t need = X[0].dtype == TS_F64 ? batch_bytes<double>(count, X, P->S)
                                           : batch_bytes<float>(count, X, P->S);
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255))
    return fail(TS_ERR_WORKSPACE, "ts_batch_prepare: need %zu bytes of 256-aligned workspace",
                need);
  P->count = count;
  P->N = N;
  P->sweeps = sweeps;
  P->dtype = X[0].dtype;
  P->solve = opt->solve;
  P->fp64 = P->S[0].fp64solve;
  TS_CUDA(cudaGetDevice(&P->device));
  P->X.assign(X, X + count);
  P->cores.assign(cores, cores + count);
  P->factors.assign(factors, factors + (size_t)count * N);
  P->flags.assign(count, nullptr);
  P->fitQ.assign(count, nullptr);
  P->fitacc.assign(count, nullptr);
  cudaStream_t st = (cudaStream_t)stream;
  char* ws = static_cast<char*>(workspace);
  TS_TRY(P->dtype == TS_F64 ? batch_prepare_impl<double>(*P, *opt, ws, st)
                            : batch_prepare_impl<float>(*P, *opt, ws, st));
  *batch_out = P.release();
  return TS_OK;
}

extern "C" ts_status ts_batch_sweeps(ts_batch batch, int32_t first, int32_t nsweeps,
                                     ts_stream stream) {
  clear_error();
  const BatchPlan* P = static_cast<const BatchPlan*>(batch);
  if (!P) return fail(TS_ERR_INVALID_ARG, "ts_batch_sweeps: NULL batch");
  if (first < 0 || nsweeps < 0 || first + nsweeps > P->sweeps)
    return fail(TS_ERR_SHAPE, "ts_batch_sweeps: sweeps [%d, %d) outside [0, %d)", first,
                first + nsweeps, P->sweeps);
  cudaStream_t st = (cudaStream_t)stream;
  return P->dtype == TS_F64 ? batch_sweeps_impl<double>(*P, first, nsweeps, st)
                            : batch_sweeps_impl<float>(*P, first, nsweeps, st);
}

extern "C" ts_status ts_batch_residuals(ts_batch batch, double* residuals, ts_stream stream) {
  clear_error();
  const BatchPlan* P = static_cast<const BatchPlan*>(batch);
  if (!P || !residuals) return fail(TS_ERR_INVALID_ARG, "ts_batch_residuals: NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  for (int i = 0; i < P->count; ++i) {
    const int N = P->N;
    if (P->dtype == TS_F64)
      TS_TRY(launch_fit_dense<double>(P->X[i], P->S[i].ranks,
                                      static_cast<const double*>(P->cores[i]),
                                      reinterpret_cast<const double* const*>(&P->factors[(size_t)i * N]),
                                      static_cast<double*>(P->fitQ[i]),
                                      static_cast<double*>(P->fitacc[i]), residuals + i, st));
    else
      TS_TRY(launch_fit_dense<float>(P->X[i], P->S[i].ranks,
                                     static_cast<const float*>(P->cores[i]),
                                     reinterpret_cast<const float* const*>(&P->factors[(size_t)i * N]),
                                     static_cast<float*>(P->fitQ[i]),
                                     static_cast<double*>(P->fitacc[i]), residuals + i, st));
  }
  return TS_OK;
}

extern "C" ts_status ts_batch_flags(ts_batch batch, int32_t* flags_out) {
  clear_error();
  const BatchPlan* P = static_cast<const BatchPlan*>(batch);
  if (!P || !flags_out) return fail(TS_ERR_INVALID_ARG, "ts_batch_flags: NULL argument");
  for (int i = 0; i < P->count; ++i)
    TS_CUDA(cudaMemcpy(flags_out + i, P->flags[i], sizeof(int32_t), cudaMemcpyDeviceToHost));
  return TS_OK;
}

extern "C" ts_status ts_batch_tiles(ts_batch batch, int32_t* tiles_out, float* ms_out) {
  clear_error();
  const BatchPlan* P = static_cast<const BatchPlan*>(batch);
  if (!P || !tiles_out) return fail(TS_ERR_INVALID_ARG, "ts_batch_tiles: NULL argument");
  for (int n = 0; n < P->N; ++n) {
    tiles_out[n] = P->tile[n];
    if (ms_out) {
      ms_out[2 * n] = P->tile_ms[n][0];
      ms_out[2 * n + 1] = P->tile_ms[n][1];
    }
  }
  return TS_OK;
}

extern "C" void ts_batch_destroy(ts_batch batch) { delete static_cast<BatchPlan*>(batch); }
