// The sketched Gram products of Alg. 5 in the BF16 precision form: C (M x N, FP32) =
// A (M x K) B (N x K)^T with A and B rounded to BF16, both K-major (rows contiguous
// along K), on the fifth-generation tensor cores with FP32 accumulation in tensor
// memory.  In the decomposition A = Z^T and B = [Z | Y Omega | Y]^T, so one launch forms
// [Z^T Z | Z^T Y Omega | Z^T Y] for a subproblem.
//
// One CTA computes a 128 x 128 tile over a range of K (split-K; the partial tiles are
// summed in split order by a second kernel, so the result is deterministic):
//   warp 0, lane 0  streams 128 x 64 BF16 tiles of A and B with TMA tensor loads
//                   (128-byte swizzle) into a 4-stage ring (full / empty mbarriers);
//   warp 1, lane 0  issues tcgen05.mma (kind::f16, BF16 in, FP32 accumulate, M = 128,
//                   N = 128, K = 16 per instruction) from shared-memory descriptors and
//                   releases each stage with tcgen05.commit;
//   all 4 warps     read the accumulator from tensor memory (tcgen05.ld, warp w owns
//                   rows 32w .. 32w + 31) and store it.
// Every wait is bounded by time; on expiry the kernel writes TS_ERR_TIMEOUT to the
// caller's flag and still releases its tensor memory.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace ts {

namespace {
constexpr int kBM = 128, kBN = 128, kBK = 64;  // kBK BF16 = one 128-byte swizzle row
constexpr int kStages = 4;
constexpr int kThreads = 128;
constexpr int kTmemCols = 128;  // FP32 accumulator columns (= kBN)
constexpr unsigned kTileBytes = kBM * kBK * 2;  // 16 KB, also for B (kBN = kBM)
constexpr unsigned long long kWaitNs = 200ull * 1000 * 1000;
}  // namespace

struct GramArgs {
  int M, N, K;
  int kb_per_split;  // K blocks (of kBK) per split
  float* out;        // splits > 1: split-major M x N partials; else C
  long ldo;          // row stride of out
  long split_stride; // elements between consecutive splits' partials (0: one split)
  int* flag;
};

__device__ __forceinline__ unsigned s_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long ns_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool bar_try(unsigned mbar, unsigned parity) {
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

__device__ __forceinline__ bool bar_wait(unsigned mbar, unsigned parity) {
  if (bar_try(mbar, parity)) return true;
  const unsigned long long t0 = ns_now();
  while (!bar_try(mbar, parity))
    if (ns_now() - t0 > kWaitNs) return false;
  return true;
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle: rows of 128 B
// (64 BF16), 8-row atoms of 1024 B stacked along M/N (stride byte offset 1024), the
// leading byte offset unused for this layout (1), descriptor version 1, swizzle mode 2.
__device__ __forceinline__ unsigned long long sw128_desc(unsigned saddr) {
  unsigned long long d = (unsigned long long)((saddr & 0x3FFFFu) >> 4);
  d |= 1ull << 16;
  d |= (unsigned long long)(1024u >> 4) << 32;
  d |= 1ull << 46;
  d |= 2ull << 61;
  return d;
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16 (bits 7-9 and
// 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr unsigned mma_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(kBN >> 3) << 17) |
         ((unsigned)(kBM >> 4) << 24);
}

__global__ void __launch_bounds__(kThreads) k_gram_tc(const __grid_constant__ CUtensorMap mapA,
                                                      const __grid_constant__ CUtensorMap mapB,
                                                      GramArgs g) {
  pdl_trigger();
  pdl_wait();
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long full_bar[kStages], empty_bar[kStages], done_bar;
  __shared__ unsigned tmem_slot;
  __shared__ int aborted, loads_issued, loads_consumed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * kBN, m0 = blockIdx.y * kBM;
  const int nkb_all = (g.K + kBK - 1) / kBK;
  const int kb0 = blockIdx.z * g.kb_per_split;
  const int nkb = max(0, min(nkb_all, kb0 + g.kb_per_split) - kb0);
  // 1024-byte aligned stage ring (the swizzle atoms must start on 1024 B)
  const unsigned ring = (s_addr(smem_raw) + 1023u) & ~1023u;

  if (threadIdx.x == 0) {
    aborted = 0;
    loads_issued = 0;
    loads_consumed = 0;
    for (int s = 0; s < kStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_addr(&full_bar[s])) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_addr(&empty_bar[s])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_addr(&done_bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     s_addr(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    for (int i = 0; i < nkb; ++i) {
      const int s = i % kStages;
      if (i >= kStages && !bar_wait(s_addr(&empty_bar[s]), (unsigned)((i / kStages - 1) & 1))) {
        atomicExch(&aborted, 1);
        break;
      }
      const unsigned sa = ring + s * 2 * kTileBytes, sb = sa + kTileBytes;
      const unsigned fb = s_addr(&full_bar[s]);
      const int kx = (kb0 + i) * kBK;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                   "r"(2 * kTileBytes)
                   : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
          "[%0], [%1, {%2, %3}], [%4];" ::"r"(sa),
          "l"(&mapA), "r"(kx), "r"(m0), "r"(fb)
          : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
          "[%0], [%1, {%2, %3}], [%4];" ::"r"(sb),
          "l"(&mapB), "r"(kx), "r"(n0), "r"(fb)
          : "memory");
      loads_issued = i + 1;
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    const unsigned idesc = mma_idesc();
    for (int i = 0; i < nkb; ++i) {
      const int s = i % kStages;
      if (!bar_wait(s_addr(&full_bar[s]), (unsigned)((i / kStages) & 1))) {
        atomicExch(&aborted, 1);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned sa = ring + s * 2 * kTileBytes, sb = sa + kTileBytes;
#pragma unroll
      for (int kk = 0; kk < kBK / 16; ++kk) {
        const unsigned long long da = sw128_desc(sa + 32u * kk), db = sw128_desc(sb + 32u * kk);
        const unsigned acc = (i > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(acc)
            : "memory");
      }
      // the stage is free once these products have read it
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              s_addr(&empty_bar[s]))
          : "memory");
      loads_consumed = i + 1;
    }
    // arrives when every product issued above has completed
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            s_addr(&done_bar))
        : "memory");
  }
  __syncwarp();

  // ---------------- epilogue: tensor memory -> registers -> global
  // (warp-uniform decisions: tcgen05.ld is issued by all 32 lanes or by none)
  bool done = bar_wait(s_addr(&done_bar), 0u);
  done = __all_sync(0xffffffffu, done);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int row = m0 + warp * 32 + lane;
  float* out = g.out + (long)blockIdx.z * g.split_stride;
  const int ab = __shfl_sync(0xffffffffu, *(volatile int*)&aborted, 0);
  const bool ok = done && !ab;
  for (int c0 = 0; c0 < kBN; c0 += 8) {
    unsigned v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (ok && nkb > 0) {
      const unsigned ta = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7])
          : "r"(ta)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    }
    if (row < g.M) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int col = n0 + c0 + j;
        if (col < g.N) out[(long)row * g.ldo + col] = __uint_as_float(v[j]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0 && aborted) {
    // loads issued but never consumed must land before the shared memory goes away
    for (int i = loads_consumed; i < loads_issued; ++i)
      bar_wait(s_addr(&full_bar[i % kStages]), (unsigned)((i / kStages) & 1));
  }
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols)
                 : "memory");
  if (threadIdx.x == 0 && (!done || aborted) && g.flag) atomicExch(g.flag, (int)TS_ERR_TIMEOUT);
}

// dst (rows x ld, BF16, row-major) <- src element (i, k) at src[i rs + k cs], k < K;
// columns K .. ld-1 are zero.  32 x 32 tiles through shared memory, so that both the
// read (along the source's contiguous index) and the write (along k) are coalesced.
__global__ void __launch_bounds__(256) k_pack_bf16(const float* __restrict__ src, long rs,
                                                   long cs, int rows, int K, int ld,
                                                   __nv_bfloat16* __restrict__ dst) {
  __shared__ float tile[32][33];
  const int i0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  const bool k_fast = cs == 1;
  for (int u = ty; u < 32; u += 8) {
    // load: coalesced along k when k is contiguous, else along i
    const int i = k_fast ? i0 + u : i0 + tx, k = k_fast ? k0 + tx : k0 + u;
    float v = 0.f;
    if (i < rows && k < K) v = src[(long)i * rs + (long)k * cs];
    if (k_fast) tile[u][tx] = v;
    else tile[tx][u] = v;
  }
  __syncthreads();
  for (int u = ty; u < 32; u += 8) {
    const int i = i0 + u, k = k0 + tx;
    if (i < rows && k < ld) dst[(long)i * ld + k] = __float2bfloat16_rn(tile[u][tx]);
  }
}

// ---------------------------------------------------------------- host side

int gram_tc_ld(int K) { return (K + 7) & ~7; }

ts_status pack_bf16(const float* src, long rs, long cs, int rows, int K, void* dst,
                    cudaStream_t st) {
  if (rows <= 0) return TS_OK;
  const int ld = gram_tc_ld(K);
  dim3 grid(ceil_div(ld, 32), ceil_div(rows, 32));
  k_pack_bf16<<<grid, 256, 0, st>>>(src, rs, cs, rows, K, ld,
                                    static_cast<__nv_bfloat16*>(dst));
  TS_LAUNCH_CHECK();
  return TS_OK;
}

ts_status gram_tc_map(const void* base, int rows, int K, CUtensorMap* map) {
  if (((uintptr_t)base & 15) != 0) return fail(TS_ERR_INVALID_ARG, "gram: BF16 operand not 16-byte aligned");
  EncodeTiledFn encode;
  TS_TRY(encode_fn(&encode));
  const int ld = gram_tc_ld(K);
  const cuuint64_t gdim[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t gstride[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)kBM};
  const cuuint32_t estride[2] = {1, 1};
  CUresult cr = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), gdim,
                       gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return fail(TS_ERR_CUDA, "gram: cuTensorMapEncodeTiled failed (%d)", (int)cr);
  return TS_OK;
}

int gram_tc_splits(int M, int N, int K) {
  const int tiles = ceil_div(M, kBM) * ceil_div(N, kBN);
  const int nkb = ceil_div(K > 0 ? K : 1, kBK);
  // at least four K blocks per split: the 4-stage ring fills, and fewer partials to add
  int splits = ceil_div(152, tiles);
  if (splits > ceil_div(nkb, 4)) splits = ceil_div(nkb, 4);
  if (splits > 32) splits = 32;
  return splits < 1 ? 1 : splits;
}

size_t gram_tc_partial_elems(int M, int N, int K) {
  const int splits = gram_tc_splits(M, N, K);
  return splits > 1 ? (size_t)splits * M * N : 0;
}

ts_status gram_tc(const CUtensorMap& mapA, const CUtensorMap& mapB, int M, int N, int K,
                  float* C, long ldc, float* partial, int* flag, cudaStream_t st) {
  if (M <= 0 || N <= 0) return TS_OK;
  int splits = gram_tc_splits(M, N, K);
  const int nkb = ceil_div(K > 0 ? K : 1, kBK);
  const int per = ceil_div(nkb, splits);
  splits = ceil_div(nkb, per);
  GramArgs g{};
  g.M = M;
  g.N = N;
  g.K = K;
  g.kb_per_split = per;
  g.flag = flag;
  if (splits > 1) {
    g.out = partial;
    g.ldo = N;
    g.split_stride = (long)M * N;
  } else {
    g.out = C;
    g.ldo = ldc;
    g.split_stride = 0;
  }
  const size_t smem = (size_t)kStages * 2 * kTileBytes + 1024;
  TS_TRY(ensure_dynamic_smem((const void*)k_gram_tc, smem));
  dim3 grid(ceil_div(N, kBN), ceil_div(M, kBM), splits);
  TS_TRY(launch_pdl(k_gram_tc, grid, dim3(kThreads), smem, st, mapA, mapB, g));
  if (splits > 1) TS_TRY(launch_split_reduce<float>(M, N, splits, partial, C, ldc, st));
  return TS_OK;
}

}  // namespace ts

using namespace ts;

// ================================================================ C ABI

extern "C" size_t ts_gram_bf16_scratch_bytes(int32_t M, int32_t N, int32_t K) {
  if (M < 1 || N < 1 || K < 1) return 0;
  Bump b;
  b.take<int>(64);
  b.take<__nv_bfloat16>((size_t)M * gram_tc_ld(K));
  b.take<__nv_bfloat16>((size_t)N * gram_tc_ld(K));
  b.take<float>(gram_tc_partial_elems(M, N, K));
  return b.off;
}

extern "C" ts_status ts_gram_bf16(int32_t M, int32_t N, int32_t K, const void* A, const void* B,
                                  void* C_out, void* scratch, size_t scratch_bytes,
                                  ts_stream stream) {
  clear_error();
  if (M < 1 || N < 1 || K < 1) return fail(TS_ERR_SHAPE, "ts_gram_bf16: need M, N, K >= 1");
  if (!A || !B || !C_out) return fail(TS_ERR_INVALID_ARG, "ts_gram_bf16: NULL argument");
  const size_t need = ts_gram_bf16_scratch_bytes(M, N, K);
  if (!scratch || scratch_bytes < need || ((uintptr_t)scratch & 255))
    return fail(TS_ERR_WORKSPACE, "ts_gram_bf16: need %zu bytes of 256-aligned scratch", need);
  cudaStream_t st = (cudaStream_t)stream;
  Bump b{static_cast<char*>(scratch)};
  int* flag = b.take<int>(64);
  __nv_bfloat16* Ab = b.take<__nv_bfloat16>((size_t)M * gram_tc_ld(K));
  __nv_bfloat16* Bb = b.take<__nv_bfloat16>((size_t)N * gram_tc_ld(K));
  float* part = b.take<float>(gram_tc_partial_elems(M, N, K));
  TS_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
  TS_TRY(pack_bf16(static_cast<const float*>(A), K, 1, M, K, Ab, st));
  TS_TRY(pack_bf16(static_cast<const float*>(B), K, 1, N, K, Bb, st));
  CUtensorMap ma, mb;
  TS_TRY(gram_tc_map(Ab, M, K, &ma));
  TS_TRY(gram_tc_map(Bb, N, K, &mb));
  return gram_tc(ma, mb, M, N, K, static_cast<float*>(C_out), N, part, flag, st);
}
