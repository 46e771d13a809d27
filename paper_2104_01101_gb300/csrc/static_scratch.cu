// tensorsketch_apply_static_scratch: the TensorSketch of a Kronecker chain with
// its scratch (twiddle table and factor spectra) in a fixed device array instead
// of caller-provided memory, for callers that cannot allocate device memory.
//
// The array is a file-scope __device__ object, so every GPU that loads this
// library holds kStaticScratchBytes of it until the process exits.  In host code
// its name is only a host-side stand-in; the device address is fetched once per
// device with cudaGetSymbolAddress (with that device current) and cached.  The cache
// is keyed by device ordinal and never invalidated: it assumes the primary context is
// not reset (cudaDeviceReset reloads the module, and the cached address may then be
// stale).  Looking the address up on every call would survive a reset but could not
// run inside a stream capture, which the cached form can.
#include <mutex>

#include "internal.cuh"

namespace ts {

constexpr size_t kStaticScratchBytes = (size_t)8 << 20;  // 8 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxStaticDevices = 64;
static void* g_static_addr[kMaxStaticDevices] = {};
static std::mutex g_static_mu;

// Device address of g_static_scratch on the current device (looked up on first use).
static ts_status static_scratch_address(void** out) {
  int dev = -1;
  TS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxStaticDevices)
    return fail(TS_ERR_UNSUPPORTED, "static scratch: device ordinal %d >= %d", dev,
                kMaxStaticDevices);
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (!g_static_addr[dev]) {
    void* p = nullptr;
    TS_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
    g_static_addr[dev] = p;
  }
  *out = g_static_addr[dev];
  return TS_OK;
}

}  // namespace ts

using namespace ts;

extern "C" size_t tensorsketch_apply_static_scratch_capacity(void) { return kStaticScratchBytes; }

extern "C" ts_status tensorsketch_apply_static_scratch(int32_t nf, const void* const* factors,
                                                       const int64_t* rows, const int32_t* cols,
                                                       const int32_t* const* tables, int32_t m,
                                                       int32_t dtype, void* Z_out,
                                                       ts_stream stream) {
  clear_error();
  if (nf >= 1 && nf < TS_MAX_ORDER && cols && m >= 1) {
    const size_t need = tensorsketch_apply_scratch_bytes(nf, cols, m, dtype);
    if (need > kStaticScratchBytes)
      return fail(TS_ERR_WORKSPACE,
                  "tensorsketch_apply_static_scratch: this problem needs %zu bytes of scratch, "
                  "more than the fixed %zu-byte device array; use tensorsketch_apply",
                  need, kStaticScratchBytes);
  }
  void* scratch = nullptr;
  TS_TRY(static_scratch_address(&scratch));
  // Every scratch element the kernels read is written earlier in the same call
  // (twiddles, then full spectra columns), so the array needs no clearing.
  return tensorsketch_apply(nf, factors, rows, cols, tables, m, dtype, Z_out, scratch,
                            kStaticScratchBytes, stream);
}
