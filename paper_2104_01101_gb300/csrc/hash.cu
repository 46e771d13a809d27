// Random objects of the method: hash tables (Sec. 3.1) and Gaussian matrices
// (Sec. 5 composite sketch, Alg. 5 test matrix), plus the library's error state.
#include <stdarg.h>
#include <stdio.h>

#include <atomic>
#include <map>
#include <mutex>
#include <utility>

#include "internal.cuh"

namespace ts {

static thread_local char g_err[1024] = {0};

ts_status fail(ts_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

void clear_error() { g_err[0] = 0; }

static std::atomic<uint64_t> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

ts_status ensure_dynamic_smem(const void* fn, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> granted;
  if (bytes > 227 * 1024)
    return fail(TS_ERR_SHAPE, "shared-memory footprint %zu bytes exceeds 227 KB", bytes);
  int dev = 0;
  TS_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  size_t& have = granted[{dev, fn}];
  if (bytes > have) {
    TS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    have = bytes;
  }
  return TS_OK;
}

// table_out[i] = bucket (poly2(i) mod nbins) | sign bit (poly3(i) odd).
__global__ void k_hash_table(HashCoefs h, int64_t size, int nbins, int32_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < size;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t x = (uint64_t)i;
    uint32_t bin = (uint32_t)(poly_mod_p(h.a, 3, x) % (uint64_t)nbins);
    bool neg = (poly_mod_p(h.b, 4, x) & 1ull) != 0;
    out[i] = pack_entry(bin, neg);
  }
}

ts_status launch_hash_table(uint64_t seed, int purpose, int sweep, int n, int k, int64_t size,
                            int nbins, int32_t* out, cudaStream_t st) {
  if (size <= 0) return TS_OK;
  HashCoefs h = hash_coefs(seed, purpose, sweep, n, k);
  int blocks = (int)((size + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  k_hash_table<<<blocks, 256, 0, st>>>(h, size, nbins, out);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

template <typename T>
__global__ void k_gaussian(uint64_t key, int64_t count, double scale, T* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = (T)(scale * gauss01(key, (uint64_t)e));
}

template <typename T>
ts_status launch_gaussian(uint64_t seed, uint64_t tag, int64_t count, double scale, T* out,
                          cudaStream_t st) {
  if (count <= 0) return TS_OK;
  // Small blocks spread the (slow) FP64 transcendental work over many SMs.
  int blocks = (int)((count + 63) / 64);
  if (blocks > 8192) blocks = 8192;
  k_gaussian<T><<<blocks, 64, 0, st>>>(object_key(seed, tag), count, scale, out);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

// Test matrices of Alg. 5 for a run of sweeps, every mode in one launch.  Mode n's block
// starts at ob.off[n] (blocks contiguous, in mode order) and is s_n x (nsweeps k_n)
// row-major: element (j, t k_n + c) is draw j k_n + c of the object
// (seed, RSVD_GAUSS, sweep0 + t, n, 0), i.e. entry (j, c) of Omega(sweep0 + t, n).
template <typename T>
__global__ void k_omegas(uint64_t seed, OmegaBlocks ob, T* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ob.total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int n = 0;
    while (n + 1 < ob.N && e >= ob.off[n + 1]) ++n;
    const int k = ob.k[n];
    const int64_t width = (int64_t)ob.nsweeps * k;
    const int64_t loc = e - ob.off[n];
    const int64_t j = loc / width;
    const int rem = (int)(loc - j * width);
    const int t = rem / k, c = rem - t * k;
    const uint64_t key = object_key(seed, make_tag(TS_PURPOSE_RSVD_GAUSS, ob.sweep0 + t, n, 0));
    out[e] = (T)gauss01(key, (uint64_t)(j * k + c));
  }
}

template <typename T>
ts_status launch_omegas(uint64_t seed, const OmegaBlocks& ob, T* out, cudaStream_t st) {
  if (ob.total <= 0) return TS_OK;
  int blocks = (int)((ob.total + 127) / 128);
  if (blocks > 8192) blocks = 8192;
  k_omegas<T><<<blocks, 128, 0, st>>>(seed, ob, out);
  TS_LAUNCH_CHECK();
  return TS_OK;
}

template ts_status launch_omegas<float>(uint64_t, const OmegaBlocks&, float*, cudaStream_t);
template ts_status launch_omegas<double>(uint64_t, const OmegaBlocks&, double*, cudaStream_t);

ts_status encode_fn(EncodeTiledFn* out) {
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

template ts_status launch_gaussian<float>(uint64_t, uint64_t, int64_t, double, float*,
                                          cudaStream_t);
template ts_status launch_gaussian<double>(uint64_t, uint64_t, int64_t, double, double*,
                                           cudaStream_t);

}  // namespace ts

using namespace ts;

extern "C" const char* ts_last_error(void) { return g_err; }

extern "C" const char* ts_version(void) { return "tsketch 0.1 (sm_103a)"; }

extern "C" uint64_t ts_kernel_launches(void) { return g_launches.load(); }

extern "C" ts_status ts_hash_table(uint64_t seed, int32_t purpose, int32_t sweep, int32_t n,
                                   int32_t k, int64_t size, int32_t nbins, int32_t* table_out,
                                   ts_stream stream) {
  clear_error();
  if (!table_out) return fail(TS_ERR_INVALID_ARG, "ts_hash_table: table_out is NULL");
  if (size < 0 || size >= (int64_t)kP31)
    return fail(TS_ERR_INVALID_ARG, "ts_hash_table: size %lld outside [0, 2^31-1)",
                (long long)size);
  if (nbins < 1) return fail(TS_ERR_INVALID_ARG, "ts_hash_table: nbins %d < 1", nbins);
  if (purpose < 0 || purpose > 255 || n < 0 || n > 255 || k < 0 || k > 255 || sweep < 0 ||
      sweep >= (1 << 24))
    return fail(TS_ERR_INVALID_ARG, "ts_hash_table: tag field out of range");
  return launch_hash_table(seed, purpose, sweep, n, k, size, nbins, table_out,
                           (cudaStream_t)stream);
}
