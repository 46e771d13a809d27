// One-pass sketch of a dense order-3 FP32 tensor (Alg. 4, right-hand sides) at
// HBM speed.  Every output Y_n[b, i_n] gathers ~s^2/m entries from all over the
// tensor, so no CTA can own an output row; the kernel therefore reads the tensor
// once in TB2 x TB3 tiles (TMA tensor loads into a multi-stage shared-memory ring)
// and pushes each tile's contributions to the L2-resident sketches with TMA bulk
// reductions of whole tile rows:
//   mode 3  Y3[H31(i1) + H32(i2), i3-range] += S(i1,i2) * T[i1, i2, i3-range]   (tile rows)
//   mode 2  Y2[H21(i1) + H23(i3), i2-range] += S(i1,i3) * T[i1, i2-range, i3]   (tile columns,
//           transposed and signed in shared memory first)
//   mode 1  Y1[H12(i2) + H13(i3), i1]       += S(i2,i3) * T[i1, i2, i3]         (shared-memory
//           buckets of the current slice i1, flushed when i1 changes)
// A CTA walks a contiguous range of tiles (slice-major), so a slice's mode-1 buckets
// are flushed at most twice per CTA.  All waits are bounded: on a timeout the kernel
// records TS_ERR_TIMEOUT in the caller's flag, drains its own bulk operations and exits.
#include <cuda.h>

#include "internal.cuh"

namespace ts {

namespace {
constexpr int kStages = 3;
constexpr int kThreads = 256;
constexpr unsigned kSpinLimit = 1u << 24;
}  // namespace

struct Dense3Sketch {
  int s1, s2, s3;
  int TB2, TB3;            // tile rows (mode 2) and columns (mode 3)
  int tiles2, tiles3;      // tiles per slice along modes 2 and 3
  long ntiles;
  float* Y1; int m1; const int32_t* t12; const int32_t* t13;   // Y1 may be null
  float* Y2; int m2; const int32_t* t21; const int32_t* t23;   // Y2 may be null
  float* Y3; int m3; const int32_t* t31; const int32_t* t32;   // Y3 may be null
  int* flag;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity) {
  for (unsigned it = 0; it < kSpinLimit; ++it) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_tile(const CUtensorMap* map, unsigned dst, unsigned mbar,
                                              int c3, int c2, int c1, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(map), "r"(c3), "r"(c2), "r"(c1), "r"(mbar)
      : "memory");
}

__device__ __forceinline__ void bulk_reduce_add(float* gdst, unsigned ssrc, unsigned bytes) {
  asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.f32 [%0], [%1], %2;" ::"l"(
                   gdst),
               "r"(ssrc), "r"(bytes)
               : "memory");
}

// Row stride of the transposed tile: a multiple of 4 floats (16-byte aligned rows for
// the bulk reductions) with stride/4 odd, so that a warp's 8 x 4 store pattern covers
// all 32 banks.
__host__ __device__ __forceinline__ int transposed_stride(int TB2) {
  const int l = TB2 + 4;
  return ((l / 4) & 1) ? l : l + 4;
}

__device__ __forceinline__ int add_mod(int a, int b, int m) {
  const int s = a + b;
  return s >= m ? s - m : s;
}

__global__ void __launch_bounds__(kThreads) k_sketch_dense3_tma(const __grid_constant__ CUtensorMap tmap,
                                                                 Dense3Sketch d) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int TB2 = d.TB2, TB3 = d.TB3;
  const int tile_elems = TB2 * TB3;
  const int ldt = transposed_stride(TB2);
  // layout: stages | 2 transposed tiles | mode-1 buckets | tables
  float* stage = reinterpret_cast<float*>(smem_raw);
  float* tbuf = stage + kStages * tile_elems;
  float* acc1 = tbuf + 2 * TB3 * ldt;
  int* h12 = reinterpret_cast<int*>(acc1 + (d.Y1 ? d.m1 : 0));
  int* h13 = h12 + d.s2;
  int* h23 = h13 + d.s3;
  int* h32 = h23 + d.s3;
  __shared__ __align__(8) unsigned long long mbar[kStages];
  __shared__ int timed_out;

  // contiguous tile range of this CTA
  const long per = (d.ntiles + gridDim.x - 1) / gridDim.x;
  const long t_begin = blockIdx.x * per;
  const long t_end = min(d.ntiles, t_begin + per);
  if (t_begin >= t_end) return;
  const int tiles_per_slice = d.tiles2 * d.tiles3;

  // tables with buckets already reduced modulo their sketch size
  auto reduced = [](int32_t e, int m) { return (int)(entry_bin(e) % m) | (e & (int)0x80000000); };
  for (int i = threadIdx.x; i < d.s2; i += blockDim.x) {
    if (d.Y1) h12[i] = reduced(d.t12[i], d.m1);
    if (d.Y3) h32[i] = reduced(d.t32[i], d.m3);
  }
  for (int i = threadIdx.x; i < d.s3; i += blockDim.x) {
    if (d.Y1) h13[i] = reduced(d.t13[i], d.m1);
    if (d.Y2) h23[i] = reduced(d.t23[i], d.m2);
  }
  if (d.Y1)
    for (int i = threadIdx.x; i < d.m1; i += blockDim.x) acc1[i] = 0.f;
  if (threadIdx.x == 0) {
    timed_out = 0;
    for (int s = 0; s < kStages; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const unsigned tile_bytes = (unsigned)tile_elems * 4u;
  auto coords = [&](long t, int& i1, int& r0, int& c0) {
    i1 = (int)(t / tiles_per_slice);
    const int w = (int)(t % tiles_per_slice);
    r0 = (w / d.tiles3) * TB2;
    c0 = (w % d.tiles3) * TB3;
  };
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages - 1; ++s) {
      const long t = t_begin + s;
      if (t >= t_end) break;
      int i1, r0, c0;
      coords(t, i1, r0, c0);
      tma_load_tile(&tmap, smem_u32(stage + s * tile_elems), smem_u32(&mbar[s]), c0, r0, i1,
                    tile_bytes);
    }
  }

  int cur_i1 = -1;
  unsigned phase_bits = 0;  // parity per stage
  for (long t = t_begin; t < t_end; ++t) {
    const int sidx = (int)((t - t_begin) % kStages);
    float* tile = stage + sidx * tile_elems;
    float* tb = tbuf + ((t - t_begin) & 1) * TB3 * ldt;
    int i1, r0, c0;
    coords(t, i1, r0, c0);
    const bool ok = mbar_wait(smem_u32(&mbar[sidx]), (phase_bits >> sidx) & 1u);
    phase_bits ^= 1u << sidx;
    if (!ok) atomicExch(&timed_out, 1);
    if (__syncthreads_or(!ok)) break;

    if (d.Y1 && i1 != cur_i1) {  // new slice: flush the previous slice's buckets
      if (cur_i1 >= 0) {
        for (int b = threadIdx.x; b < d.m1; b += blockDim.x) {
          const float v = acc1[b];
          if (v != 0.f) atomicAdd(d.Y1 + (long)b * d.s1 + cur_i1, v);
          acc1[b] = 0.f;
        }
        __syncthreads();
      }
    }
    cur_i1 = i1;
    // per-element work: mode-1 buckets, transposed+signed copy (mode 2), in-place sign (mode 3)
    int h21 = 0, h31 = 0;
    bool n21 = false, n31 = false;
    if (d.Y2) { const int e = d.t21[i1]; h21 = entry_bin(e) % d.m2; n21 = entry_neg(e); }
    if (d.Y3) { const int e = d.t31[i1]; h31 = entry_bin(e) % d.m3; n31 = entry_neg(e); }
    // Micro-blocks of 8 columns x 4 rows per warp instruction: the transposed store
    // (row stride ldt = TB2 + 4) then hits 32 distinct banks.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nqc = TB3 / 8, nmb = nqc * (TB2 / 4);
    for (int mb = warp; mb < nmb; mb += (int)(blockDim.x >> 5)) {
      const int cc = (mb % nqc) * 8 + (lane >> 2);
      const int rr = (mb / nqc) * 4 + (lane & 3);
      const int i2 = r0 + rr, i3 = c0 + cc;
      const float v = tile[rr * TB3 + cc];
      if (d.Y1) {
        const int a = h12[i2], b = h13[i3];
        const int bin = add_mod(entry_bin(a), entry_bin(b), d.m1);
        if (v != 0.f) atomicAdd(&acc1[bin], (entry_neg(a) ^ entry_neg(b)) ? -v : v);
      }
      if (d.Y2) tb[cc * ldt + rr] = (n21 ^ entry_neg(h23[i3])) ? -v : v;
      if (d.Y3 && (n31 ^ entry_neg(h32[i2]))) tile[rr * TB3 + cc] = -v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (warp == 0) {  // every lane issues and tracks its own share of the bulk reductions
      if (d.Y3)
        for (int rr = lane; rr < TB2; rr += 32) {
          const int b = add_mod(h31, entry_bin(h32[r0 + rr]), d.m3);
          bulk_reduce_add(d.Y3 + (long)b * d.s3 + c0, smem_u32(tile + rr * TB3), TB3 * 4u);
        }
      if (d.Y2)
        for (int cc = lane; cc < TB3; cc += 32) {
          const int b = add_mod(h21, entry_bin(h23[c0 + cc]), d.m2);
          bulk_reduce_add(d.Y2 + (long)b * d.s2 + r0, smem_u32(tb + cc * ldt), TB2 * 4u);
        }
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      // the stage refilled next was read by the previous tile's reductions
      asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
    }
    __syncwarp();
    if (threadIdx.x == 0) {
      const long tn = t + kStages - 1;
      if (tn < t_end) {
        const int sn = (int)((tn - t_begin) % kStages);
        int ni1, nr0, nc0;
        coords(tn, ni1, nr0, nc0);
        tma_load_tile(&tmap, smem_u32(stage + sn * tile_elems), smem_u32(&mbar[sn]), nc0, nr0,
                      ni1, tile_bytes);
      }
    }
    __syncthreads();
  }
  if ((threadIdx.x >> 5) == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  if (timed_out) {
    if (threadIdx.x == 0) {
      if (d.flag) atomicExch(d.flag, (int)TS_ERR_TIMEOUT);
      // let the tile loads still in flight land before the block's shared memory goes away
      for (int s = 0; s < kStages; ++s) mbar_wait(smem_u32(&mbar[s]), (phase_bits >> s) & 1u);
    }
    __syncthreads();
    return;
  }
  if (d.Y1 && cur_i1 >= 0) {
    __syncthreads();
    for (int b = threadIdx.x; b < d.m1; b += blockDim.x) {
      const float v = acc1[b];
      if (v != 0.f) atomicAdd(d.Y1 + (long)b * d.s1 + cur_i1, v);
    }
  }
}

// ---------------------------------------------------------------- host side

// Largest divisor of s that is a multiple of `step` and at most `cap` (0 if none).
static int tile_divisor(long s, int cap, int step) {
  for (int t = cap - cap % step; t >= step; t -= step)
    if (s % t == 0) return t;
  return 0;
}
static int tile_rows(long s2) { return tile_divisor(s2, 80, 4); }
static int tile_cols(long s3) { return tile_divisor(s3, 80, 8); }

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                   const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                   const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static ts_status encode_fn(EncodeTiledFn* out) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    TS_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p)
      return fail(TS_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  *out = fn;
  return TS_OK;
}

bool dense3_tma_eligible(const ts_tensor& X, const SketchJob* jobs, int njobs) {
  if (X.format != TS_DENSE || X.dtype != TS_F32 || X.order != 3) return false;
  if (((uintptr_t)X.values & 15) != 0) return false;
  if (tile_rows(X.dims[1]) == 0 || tile_cols(X.dims[2]) == 0) return false;
  bool seen[3] = {false, false, false};
  for (int j = 0; j < njobs; ++j) {
    const int n = jobs[j].mode;
    if (n < 0 || n > 2 || seen[n]) return false;
    seen[n] = true;
    if (((uintptr_t)jobs[j].out & 15) != 0) return false;
  }
  return true;
}

size_t dense3_tma_smem_bytes(const ts_tensor& X, const SketchJob* jobs, int njobs) {
  const int TB2 = tile_rows(X.dims[1]), TB3 = tile_cols(X.dims[2]);
  int m1 = 0;
  for (int j = 0; j < njobs; ++j)
    if (jobs[j].mode == 0) m1 = jobs[j].nbins;
  return sizeof(float) * ((size_t)kStages * TB2 * TB3 + 2 * (size_t)TB3 * transposed_stride(TB2) +
                          m1) +
         sizeof(int) * (2 * (size_t)X.dims[1] + 2 * (size_t)X.dims[2]);
}

ts_status launch_dense3_tma(const ts_tensor& X, const SketchJob* jobs, int njobs, int* flag,
                            cudaStream_t st) {
  Dense3Sketch d{};
  d.s1 = (int)X.dims[0];
  d.s2 = (int)X.dims[1];
  d.s3 = (int)X.dims[2];
  d.TB2 = tile_rows(d.s2);
  d.TB3 = tile_cols(d.s3);
  d.tiles2 = d.s2 / d.TB2;
  d.tiles3 = d.s3 / d.TB3;
  d.ntiles = (long)d.s1 * d.tiles2 * d.tiles3;
  d.flag = flag;
  for (int j = 0; j < njobs; ++j) {
    const SketchJob& J = jobs[j];
    float* out = static_cast<float*>(J.out);
    TS_CUDA(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)J.nbins * X.dims[J.mode], st));
    if (J.mode == 0) { d.Y1 = out; d.m1 = J.nbins; d.t12 = J.tables[1]; d.t13 = J.tables[2]; }
    if (J.mode == 1) { d.Y2 = out; d.m2 = J.nbins; d.t21 = J.tables[0]; d.t23 = J.tables[2]; }
    if (J.mode == 2) { d.Y3 = out; d.m3 = J.nbins; d.t31 = J.tables[0]; d.t32 = J.tables[1]; }
  }
  EncodeTiledFn encode;
  TS_TRY(encode_fn(&encode));
  CUtensorMap map;
  const cuuint64_t gdim[3] = {(cuuint64_t)d.s3, (cuuint64_t)d.s2, (cuuint64_t)d.s1};
  const cuuint64_t gstride[2] = {(cuuint64_t)d.s3 * 4, (cuuint64_t)d.s2 * d.s3 * 4};
  const cuuint32_t box[3] = {(cuuint32_t)d.TB3, (cuuint32_t)d.TB2, 1};
  const cuuint32_t estride[3] = {1, 1, 1};
  CUresult cr = encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(X.values), gdim,
                       gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return fail(TS_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
  const size_t smem = dense3_tma_smem_bytes(X, jobs, njobs);
  TS_TRY(ensure_dynamic_smem((const void*)k_sketch_dense3_tma, smem));
  int dev = 0, nsm = 0;
  TS_CUDA(cudaGetDevice(&dev));
  TS_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  long grid = nsm;
  if (grid > d.ntiles) grid = d.ntiles;
  k_sketch_dense3_tma<<<(int)grid, kThreads, smem, st>>>(map, d);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

}  // namespace ts
