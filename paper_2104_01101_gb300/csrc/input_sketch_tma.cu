// One-pass sketch of a dense order-3 FP32 tensor (Alg. 4, right-hand sides; the
// composite sketch of Init-RRF, Sec. 5) at HBM speed.  Every output Y_n[b, i_n]
// gathers ~s^2/m entries from all over the tensor, so no CTA can own an output row;
// the kernel reads the tensor once in TB2 x TB3 tiles and sends each entry's
// contributions to the L2-resident sketches:
//   mode 3  Y3[H31(i1) + H32(i2), i3]  += S(i1,i2) T[i1,i2,i3]   (vector reductions of
//           4 consecutive i3 straight from registers)
//   mode 2  Y2[H21(i1) + H23(i3), i2]  += S(i1,i3) T[i1,i2,i3]   (4 consecutive i2 after a
//           transpose of the 16 x 16 micro-block in per-warp shared memory)
//   mode 1  Y1[H12(i2) + H13(i3), i1]  += S(i2,i3) T[i1,i2,i3]   (shared-memory buckets of
//           the current slice i1 in 32-bit fixed point, double-buffered, flushed when i1
//           changes; see below)
// Warp roles: one producer warp streams tiles with TMA tensor loads into a ring of
// shared-memory stages (full / empty mbarriers); the consumer warps split every tile
// into 16 x 16 micro-blocks.  A CTA walks a contiguous, slice-major range of tiles, so
// a slice's buckets are flushed at most twice per CTA.  Every wait is bounded by time:
// on expiry the kernel records TS_ERR_TIMEOUT in the caller's flag, the warps fall
// through the remaining tiles without computing (so the consumer barriers stay
// matched), and the producer waits, again bounded, for its loads in flight.
//
// Mode-1 buckets in fixed point.  Shared-memory float adds are a compare-and-swap loop on
// this GPU (measured: 4 lane-ops per clock per SM at random addresses, against 14.5 for
// 32-bit integer adds), so each slice's buckets accumulate integers: a value v becomes
// round(v * 2^q / B), where B is the largest |v| of the first tile of the slice that this
// CTA reads, and q (<= 22) leaves room for the largest number of entries any bucket can
// receive, bounded by min(s2 * mult(H13), s3 * mult(H12)) with mult the largest number of
// indices sharing one bucket in a table (q < 18, e.g. degenerate tables that send whole
// slices to one bucket: no fixed point, every value goes to L2 in FP32).  Integer sums are exact and independent of the
// order of the adds; the flush multiplies by B / 2^q.  Values with |v| > B (rare: larger
// than everything in the slice's first tile) are added to the sketch in L2 directly, in
// FP32.  The quantisation error of one entry is at most B 2^-(q+1).
#include <cuda.h>

#include "internal.cuh"

namespace ts {

namespace {
constexpr int kConsumers = 24;  // consumer warps
constexpr int kThreads = 32 * (kConsumers + 1);
constexpr int kMaxStages = 6;
constexpr int kTrs = 20;  // row stride of the transposed micro-block (16-byte rows)
constexpr unsigned long long kWaitNs = 200ull * 1000 * 1000;  // 200 ms per wait
}  // namespace

struct Dense3Sketch {
  int s1, s2, s3;
  int TB2, TB3;            // tile rows (mode 2) and columns (mode 3)
  int tiles2, tiles3;      // tiles per slice along modes 2 and 3
  int stages;
  long ntiles;
  float* Y1; int m1; const int32_t* t12; const int32_t* t13;   // Y1 may be null
  float* Y2; int m2; const int32_t* t21; const int32_t* t23;   // Y2 may be null
  float* Y3; int m3; const int32_t* t31; const int32_t* t32;   // Y3 may be null
  int* flag;
};

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try(unsigned mbar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of the given parity to complete; false after kWaitNs.
__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned parity) {
  if (mbar_try(mbar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try(mbar, parity))
    if (global_ns() - t0 > kWaitNs) return false;
  return true;
}

__device__ __forceinline__ void mbar_arrive(unsigned mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
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

// Y[0..3] += v[0..3] in L2 (16-byte aligned address).
__device__ __forceinline__ void red_add4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c),
               "f"(d)
               : "memory");
}

__device__ __forceinline__ int add_mod(int a, int b, int m) {
  const int s = a + b;
  return s >= m ? s - m : s;
}

// *p += v in shared memory, no return value.
__device__ __forceinline__ void red_shared_add(float* p, float v) {
  asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(smem_u32(p)), "f"(v) : "memory");
}

// *p += v in shared memory (32-bit integer add, no return value).
__device__ __forceinline__ void red_shared_add_s32(int* p, int v) {
  asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(smem_u32(p)), "r"(v) : "memory");
}

// round(x) for |x| <= 2^22: adding 1.5 * 2^23 leaves the rounded integer in the low
// mantissa bits (round-to-nearest-even of the float addition).
__device__ __forceinline__ int round_small(float x, float scale) {
  return __float_as_int(fmaf(x, scale, 12582912.0f)) - 0x4B400000;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Flip the sign of x when the sign bit of s is set.
__device__ __forceinline__ float apply_sign(float x, int s) {
  return __int_as_float(__float_as_int(x) ^ (s & (int)0x80000000));
}

// Byte offsets of the dynamic shared memory (16-byte aligned sections).
struct SmemLayout {
  size_t acc1, rowtab, coltab, scratch, total;
};
__host__ __device__ inline SmemLayout smem_layout(int stages, int tile_elems, int m1, int rows,
                                                  int cols) {
  auto up16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  SmemLayout L;
  L.acc1 = (size_t)stages * tile_elems * sizeof(float);
  L.rowtab = up16(L.acc1 + 2 * (size_t)m1 * sizeof(float));
  L.coltab = up16(L.rowtab + (size_t)rows * sizeof(int2));
  L.scratch = up16(L.coltab + (size_t)cols * sizeof(int2));
  L.total = L.scratch + (size_t)kConsumers * 16 * kTrs * sizeof(float);
  return L;
}

__global__ void __launch_bounds__(kThreads) k_sketch_dense3_tma(const __grid_constant__ CUtensorMap tmap,
                                                                 Dense3Sketch d) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long full_bar[kMaxStages], empty_bar[kMaxStages];
  __shared__ int abort_flag;
  __shared__ int q1_mult[2];    // largest bucket multiplicity of H12 and H13 (mode 1)
  __shared__ int q1_max[2];     // per bucket buffer: largest |v| bits of the slice's first tile
  const int TB2 = d.TB2, TB3 = d.TB3, S = d.stages;
  const int tile_elems = TB2 * TB3;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // layout: stages | mode-1 buckets (2 x m1) | row table | column table | scratch
  const int m1b = d.Y1 ? d.m1 : 0;
  const SmemLayout L = smem_layout(S, tile_elems, m1b, d.tiles2 * TB2, d.tiles3 * TB3);
  float* stage = reinterpret_cast<float*>(smem_raw);
  int* acc1 = reinterpret_cast<int*>(smem_raw + L.acc1);  // mode-1 buckets, fixed point
  int2* rowtab = reinterpret_cast<int2*>(smem_raw + L.rowtab);  // {H12, H32} per i2 (reduced)
  int2* coltab = reinterpret_cast<int2*>(smem_raw + L.coltab);  // {H13, H23} per i3 (reduced)
  float* scratch = reinterpret_cast<float*>(smem_raw + L.scratch);

  const long per = (d.ntiles + gridDim.x - 1) / gridDim.x;
  const long t_begin = blockIdx.x * per;
  const long t_end = min(d.ntiles, t_begin + per);
  if (t_begin >= t_end) return;
  const int ntl = (int)(t_end - t_begin);
  const int tiles_per_slice = d.tiles2 * d.tiles3;

  // hash tables with buckets reduced modulo their sketch size; padding entries are zero
  auto reduced = [](int32_t e, int m) { return (int)(entry_bin(e) % m) | (e & (int)0x80000000); };
  for (int i = tid; i < d.tiles2 * TB2; i += blockDim.x) {
    int2 v = make_int2(0, 0);
    if (i < d.s2) {
      if (d.Y1) v.x = reduced(d.t12[i], d.m1);
      if (d.Y3) v.y = reduced(d.t32[i], d.m3);
    }
    rowtab[i] = v;
  }
  for (int i = tid; i < d.tiles3 * TB3; i += blockDim.x) {
    int2 v = make_int2(0, 0);
    if (i < d.s3) {
      if (d.Y1) v.x = reduced(d.t13[i], d.m1);
      if (d.Y2) v.y = reduced(d.t23[i], d.m2);
    }
    coltab[i] = v;
  }
  for (int i = tid; i < 2 * m1b; i += blockDim.x) acc1[i] = 0;
  if (tid == 0) {
    abort_flag = 0;
    q1_mult[0] = q1_mult[1] = 0;
    q1_max[0] = q1_max[1] = 0;
    for (int s = 0; s < S; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full_bar[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty_bar[s])),
                   "r"(kConsumers)
                   : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  auto coords = [&](long t, int& i1, int& r0, int& c0) {
    i1 = (int)(t / tiles_per_slice);
    const int w = (int)(t - (long)i1 * tiles_per_slice);
    r0 = (w / d.tiles3) * TB2;
    c0 = (w - (w / d.tiles3) * d.tiles3) * TB3;
  };

  if (warp == kConsumers) {
    // ---------------- producer
    if (lane == 0) {
      const unsigned bytes = (unsigned)tile_elems * 4u;
      int issued = 0;
      for (int lt = 0; lt < ntl; ++lt) {
        const int s = lt % S;
        if (lt >= S && !mbar_wait(smem_u32(&empty_bar[s]), (unsigned)((lt / S - 1) & 1))) {
          atomicExch(&abort_flag, 1);
          break;
        }
        if (*(volatile int*)&abort_flag) break;
        int i1, r0, c0;
        coords(t_begin + lt, i1, r0, c0);
        tma_load_tile(&tmap, smem_u32(stage + (size_t)s * tile_elems), smem_u32(&full_bar[s]), c0,
                      r0, i1, bytes);
        issued = lt + 1;
      }
      // the loads still in flight must land before the block's shared memory goes away
      for (int lt = max(0, issued - S); lt < issued; ++lt)
        mbar_wait(smem_u32(&full_bar[lt % S]), (unsigned)((lt / S) & 1));
    }
  } else {
    // ---------------- consumers
    const int nmb3 = TB3 >> 4, nmb = (TB2 >> 4) * nmb3;  // 16 x 16 micro-blocks per tile
    float* tr = scratch + warp * 16 * kTrs;
    const int rq = lane >> 2, cq = lane & 3;  // load: rows rq and rq + 8, columns 4 cq .. +3
    const int tc = lane & 7, tq = lane >> 3;  // transposed read: column tc (+8), rows 4 tq .. +3
    // this lane's transposed-store offsets: element (row rq + 8h, column 4 cq + c) goes to
    // tr[col][row ^ 8 (col >> 3)]; the XOR keeps the stores and the reads conflict-free
    int st_off[2][4];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int col = 4 * cq + c, row = rq + 8 * h;
        st_off[h][c] = col * kTrs + (row ^ ((col >> 3) << 3));
      }
    // mode-1 fixed point (see the header): the precision q from the tables' bucket
    // multiplicities; the scale per slice from the first tile of the slice
    int qbits = 0;
    if (d.Y1) {
      int* hist12 = acc1;
      int* hist13 = acc1 + m1b;
      int mx12 = 0, mx13 = 0;
      for (int i = tid; i < d.s2; i += kConsumers * 32)
        mx12 = max(mx12, atomicAdd(hist12 + entry_bin(rowtab[i].x), 1) + 1);
      for (int i = tid; i < d.s3; i += kConsumers * 32)
        mx13 = max(mx13, atomicAdd(hist13 + entry_bin(coltab[i].x), 1) + 1);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        mx12 = max(mx12, __shfl_xor_sync(0xffffffffu, mx12, o));
        mx13 = max(mx13, __shfl_xor_sync(0xffffffffu, mx13, o));
      }
      if (lane == 0) {
        atomicMax(&q1_mult[0], mx12);
        atomicMax(&q1_mult[1], mx13);
      }
      asm volatile("bar.sync 1, %0;" ::"n"(kConsumers * 32) : "memory");
      for (int i = tid; i < 2 * m1b; i += kConsumers * 32) acc1[i] = 0;
      const long bound = min((long)d.s2 * q1_mult[1], (long)d.s3 * q1_mult[0]);
      qbits = 22;
      while (qbits > 0 && ((long)1 << qbits) * bound > 2147483647l) --qbits;
      if (qbits < 18) qbits = 0;  // too coarse: every value goes to L2 in FP32 instead
    }
    int buf = 0;
    float q_lim = 0.f, q_scale = 0.f, q_back = 0.f;  // this slice's fixed-point scale
    int cur_i1 = -1, h21 = 0, h31 = 0;
    bool aborted = false;
    int i1 = (int)(t_begin / tiles_per_slice);
    int w = (int)(t_begin - (long)i1 * tiles_per_slice);  // tile within the slice
    int mb0 = warp;  // first micro-block of this warp in the current tile
    // every consumer warp runs this at the start of a slice (same control flow in all)
    auto flush1 = [&](int slice, int b_, float back) {
      int* a = acc1 + b_ * m1b;
      for (int b = tid; b < d.m1; b += kConsumers * 32) {
        const int q = a[b];
        if (q != 0) atomicAdd(d.Y1 + (long)b * d.s1 + slice, (float)q * back);
        a[b] = 0;
      }
    };
    for (int lt = 0; lt < ntl; ++lt) {
      const int s = lt % S;
      const int r0 = (w / d.tiles3) * TB2, c0 = (w - (w / d.tiles3) * d.tiles3) * TB3;
      if (!aborted) {
        aborted = *(volatile int*)&abort_flag != 0;
        if (!aborted && !mbar_wait(smem_u32(&full_bar[s]), (unsigned)((lt / S) & 1))) {
          atomicExch(&abort_flag, 1);
          aborted = true;
        }
      }
      const float* tile = stage + (size_t)s * tile_elems;
      if (i1 != cur_i1) {
        if (d.Y1) {
          // all warps are done with the previous slice's buckets; reset the new slice's max
          if (tid == 0) q1_max[buf ^ 1] = 0;
          asm volatile("bar.sync 1, %0;" ::"n"(kConsumers * 32) : "memory");
          if (cur_i1 >= 0) {
            flush1(cur_i1, buf, q_back);
            buf ^= 1;
          }
          // largest |v| of this tile (the slice's first tile in this CTA's walk)
          float mx = 0.f;
          if (!aborted)
            for (int mb = mb0; mb < nmb; mb += kConsumers) {
              const int rr0 = (mb / nmb3) * 16, cc0 = (mb - (mb / nmb3) * nmb3) * 16;
              const float* tp = tile + (rr0 + rq) * TB3 + cc0 + 4 * cq;
              const float4 x0 = *reinterpret_cast<const float4*>(tp);
              const float4 x1 = *reinterpret_cast<const float4*>(tp + 8 * TB3);
              mx = fmaxf(mx, fmaxf(fmaxf(fabsf(x0.x), fabsf(x0.y)), fmaxf(fabsf(x0.z), fabsf(x0.w))));
              mx = fmaxf(mx, fmaxf(fmaxf(fabsf(x1.x), fabsf(x1.y)), fmaxf(fabsf(x1.z), fabsf(x1.w))));
            }
          mx = warp_max(mx);
          if (lane == 0) atomicMax(&q1_max[buf], __float_as_int(mx));
          asm volatile("bar.sync 1, %0;" ::"n"(kConsumers * 32) : "memory");
          const float B = __int_as_float(q1_max[buf]);
          if (qbits > 0 && B > 0.f && B < 1e30f) {
            q_lim = B;
            q_scale = (float)(1 << qbits) / B;
            q_back = B / (float)(1 << qbits);
          } else {
            q_lim = -1.f;  // no fixed point for this slice: every value goes to L2
            q_scale = 0.f;
            q_back = 0.f;
          }
        }
        cur_i1 = i1;
        if (d.Y2) h21 = reduced(d.t21[i1], d.m2);
        if (d.Y3) h31 = reduced(d.t31[i1], d.m3);
      }
      if (!aborted) {
        int* a1 = acc1 + buf * m1b;
        const int b21 = entry_bin(h21), b31 = entry_bin(h31);
        for (int mb = mb0; mb < nmb; mb += kConsumers) {
          const int rr0 = (mb / nmb3) * 16, cc0 = (mb - (mb / nmb3) * nmb3) * 16;
          const int i3 = c0 + cc0 + 4 * cq;
          const float* tp = tile + (rr0 + rq) * TB3 + cc0 + 4 * cq;
          const float4 x0 = *reinterpret_cast<const float4*>(tp);
          const float4 x1 = *reinterpret_cast<const float4*>(tp + 8 * TB3);
          const float v[2][4] = {{x0.x, x0.y, x0.z, x0.w}, {x1.x, x1.y, x1.z, x1.w}};
          const int2 rt0 = rowtab[r0 + rr0 + rq], rt1 = rowtab[r0 + rr0 + rq + 8];
          const int2 rt[2] = {rt0, rt1};
          if (d.Y1) {
            // padding rows / columns carry zero values and zero hashes: no guards needed
            const int4 ctA = *reinterpret_cast<const int4*>(coltab + i3);
            const int4 ctB = *reinterpret_cast<const int4*>(coltab + i3 + 2);
            const int c13[4] = {ctA.x, ctA.z, ctB.x, ctB.z};
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                const int b = add_mod(entry_bin(rt[h].x), entry_bin(c13[c]), d.m1);
                const float sv = apply_sign(v[h][c], rt[h].x ^ c13[c]);
                if (fabsf(sv) <= q_lim)
                  red_shared_add_s32(a1 + b, round_small(sv, q_scale));
                else
                  atomicAdd(d.Y1 + (long)b * d.s1 + i1, sv);
              }
          }
          if (d.Y3 && i3 < d.s3) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int sg = h31 ^ rt[h].y;
              float* dst = d.Y3 + (long)add_mod(b31, entry_bin(rt[h].y), d.m3) * d.s3 + i3;
              red_add4(dst, apply_sign(v[h][0], sg), apply_sign(v[h][1], sg),
                       apply_sign(v[h][2], sg), apply_sign(v[h][3], sg));
            }
          }
          if (d.Y2) {
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
              for (int c = 0; c < 4; ++c) tr[st_off[h][c]] = v[h][c];
            __syncwarp();
            const int j2 = r0 + rr0 + 4 * tq;
#pragma unroll
            for (int p = 0; p < 2; ++p) {
              const int col = tc + 8 * p;
              const float4 x = *reinterpret_cast<const float4*>(tr + col * kTrs + ((4 * tq) ^ (8 * p)));
              const int e23 = coltab[c0 + cc0 + col].y;
              const int sg = h21 ^ e23;
              if (j2 < d.s2)
                red_add4(d.Y2 + (long)add_mod(b21, entry_bin(e23), d.m2) * d.s2 + j2, apply_sign(x.x, sg),
                         apply_sign(x.y, sg), apply_sign(x.z, sg), apply_sign(x.w, sg));
            }
            __syncwarp();
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&empty_bar[s]));
      // advance: next tile of the walk, and this warp's first micro-block in it
      mb0 = (mb0 - nmb % kConsumers + kConsumers) % kConsumers;
      if (++w == tiles_per_slice) {
        w = 0;
        ++i1;
      }
    }
    if (d.Y1) {
      asm volatile("bar.sync 1, %0;" ::"n"(kConsumers * 32) : "memory");
      flush1(cur_i1, buf, q_back);
    }
  }
  __syncthreads();
  if (tid == 0 && abort_flag && d.flag) atomicExch(d.flag, (int)TS_ERR_TIMEOUT);
}

// ---------------------------------------------------------------- host side

// Tile extent along one mode: a multiple of 16 from the candidates, least padding first,
// then the larger (extents = 16 mod 32 keep the micro-block loads free of bank conflicts).
static int tile_extent(long s, const int* cand, int ncand) {
  int best = 0;
  long best_pad = 0;
  for (int i = 0; i < ncand; ++i) {
    const long pad = ceil_div(s, (long)cand[i]) * cand[i] - s;
    if (best == 0 || pad < best_pad || (pad == best_pad && cand[i] > best)) {
      best = cand[i];
      best_pad = pad;
    }
  }
  return best;
}
static const int kRowCand[] = {48, 64, 80, 96, 112};
static const int kColCand[] = {48, 80, 112};
static int tile_rows(long s2) { return s2 <= 16 ? 16 : tile_extent(s2, kRowCand, 5); }
static int tile_cols(long s3) { return s3 <= 16 ? 16 : tile_extent(s3, kColCand, 3); }

bool dense3_tma_eligible(const ts_tensor& X, const SketchJob* jobs, int njobs) {
  if (X.format != TS_DENSE || X.dtype != TS_F32 || X.order != 3) return false;
  if (((uintptr_t)X.values & 15) != 0) return false;
  if (X.dims[1] % 4 != 0 || X.dims[2] % 4 != 0) return false;  // 16-byte rows and reductions
  if (X.dims[0] >= (1l << 31) || X.dims[1] * X.dims[2] >= (1l << 31)) return false;
  bool seen[3] = {false, false, false};
  for (int j = 0; j < njobs; ++j) {
    const int n = jobs[j].mode;
    if (n < 0 || n > 2 || seen[n]) return false;
    seen[n] = true;
    if (((uintptr_t)jobs[j].out & 15) != 0) return false;
  }
  return true;
}

static int job_m1(const SketchJob* jobs, int njobs) {
  for (int j = 0; j < njobs; ++j)
    if (jobs[j].mode == 0) return jobs[j].nbins;
  return 0;
}

static SmemLayout layout_for(const ts_tensor& X, const SketchJob* jobs, int njobs, int stages) {
  const int TB2 = tile_rows(X.dims[1]), TB3 = tile_cols(X.dims[2]);
  return smem_layout(stages, TB2 * TB3, job_m1(jobs, njobs),
                     (int)(ceil_div(X.dims[1], (long)TB2) * TB2),
                     (int)(ceil_div(X.dims[2], (long)TB3) * TB3));
}

static int pick_stages(const ts_tensor& X, const SketchJob* jobs, int njobs) {
  int s = kMaxStages;
  while (s > 2 && layout_for(X, jobs, njobs, s).total + 1024 > kMaxSmem) --s;
  return s;
}

size_t dense3_tma_smem_bytes(const ts_tensor& X, const SketchJob* jobs, int njobs) {
  return layout_for(X, jobs, njobs, pick_stages(X, jobs, njobs)).total;
}

ts_status launch_dense3_tma(const ts_tensor& X, const SketchJob* jobs, int njobs, int* flag,
                            cudaStream_t st) {
  Dense3Sketch d{};
  d.s1 = (int)X.dims[0];
  d.s2 = (int)X.dims[1];
  d.s3 = (int)X.dims[2];
  d.TB2 = tile_rows(d.s2);
  d.TB3 = tile_cols(d.s3);
  d.tiles2 = (int)ceil_div((long)d.s2, (long)d.TB2);
  d.tiles3 = (int)ceil_div((long)d.s3, (long)d.TB3);
  d.ntiles = (long)d.s1 * d.tiles2 * d.tiles3;
  d.stages = pick_stages(X, jobs, njobs);
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
