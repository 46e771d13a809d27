// Shared device/host helpers of libtsketch: status plumbing, the counter-based
// generator (splitmix64, Steele-Lea-Flood 2014), the polynomial hash family over
// Z_p, p = 2^31 - 1 (Carter-Wegman), packed hash-table entries and small complex
// arithmetic.  The random objects realise the requirements of Sec. 3.1 (3-wise
// independent buckets, 4-wise independent signs), Sec. 5 (Gaussian composite
// factor) and Alg. 5 (Gaussian test matrix).
#pragma once

#include <cuda_runtime.h>
#include <utility>
#include <stdint.h>
#include <stddef.h>

#include "../../include/tsketch.h"

namespace ts {

// ---------------------------------------------------------------- status

ts_status fail(ts_status st, const char* fmt, ...);
void clear_error();

#define TS_TRY(expr)                         \
  do {                                       \
    ts_status st_ = (expr);                  \
    if (st_ != TS_OK) return st_;            \
  } while (0)

#define TS_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return ::ts::fail(TS_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                               \
  } while (0)

// Every kernel launch is followed by this: it counts the launch (ts_kernel_launches)
// and turns a launch error into TS_ERR_CUDA.
void note_launch();
#define TS_LAUNCH_CHECK()           \
  do {                              \
    ::ts::note_launch();            \
    TS_CUDA(cudaGetLastError());    \
  } while (0)

// Raise the dynamic shared-memory limit of kernel `fn` on the current device to at
// least `bytes` (cached per device and kernel; static shared memory counts against
// the default 48 KB, so every launch with dynamic shared memory goes through this).
ts_status ensure_dynamic_smem(const void* fn, size_t bytes);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Programmatic dependent launch.  A kernel launched by launch_pdl may be scheduled while
// the kernel before it in the stream is still running: pdl_trigger() at its start lets
// the next kernel launch once every block of this one has started, and pdl_wait()
// blocks until the previous kernel has completed and its writes are visible, so a
// kernel calls it before reading anything the previous one wrote.  Both are no-ops
// when the launch carried no programmatic dependency.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
ts_status launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                     cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  TS_CUDA(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
  TS_LAUNCH_CHECK();
  return TS_OK;
}

// Bump allocator over caller-provided scratch.  With base == nullptr it only
// measures, which is how every *_bytes query is answered.
struct Bump {
  char* base = nullptr;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = align_up(off, 256);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

inline int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------- random objects

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kP31 = 2147483647ull;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Key of the object named by `tag` under `seed`; element idx then draws
// mix64(key + Gamma * (idx + 1)).
__host__ __device__ __forceinline__ uint64_t object_key(uint64_t seed, uint64_t tag) {
  return mix64(seed + kGamma * (tag + 1));
}
__host__ __device__ __forceinline__ uint64_t draw64(uint64_t key, uint64_t idx) {
  return mix64(key + kGamma * (idx + 1));
}

__host__ __device__ __forceinline__ uint64_t make_tag(int purpose, int sweep, int n, int k) {
  return ((uint64_t)purpose << 56) | ((uint64_t)sweep << 32) | ((uint64_t)n << 16) | (uint64_t)k;
}

// 53-bit uniform in [0, 1).
__device__ __forceinline__ double uniform01(uint64_t key, uint64_t idx) {
  return (double)(draw64(key, idx) >> 11) * 0x1.0p-53;
}

// N(0,1) by Box-Muller from counters 2e and 2e+1 (u1 in (0,1], u2 in [0,1)).
__device__ __forceinline__ double gauss01(uint64_t key, uint64_t e) {
  double u1 = ((double)(draw64(key, 2 * e) >> 11) + 1.0) * 0x1.0p-53;
  double u2 = (double)(draw64(key, 2 * e + 1) >> 11) * 0x1.0p-53;
  return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

// Coefficients of one table: bucket polynomial a[0..2], sign polynomial b[0..3].
struct HashCoefs {
  uint64_t a[3];
  uint64_t b[4];
};

inline HashCoefs hash_coefs(uint64_t seed, int purpose, int sweep, int n, int k) {
  HashCoefs h;
  uint64_t key = object_key(seed, make_tag(purpose, sweep, n, k));
  for (int j = 0; j < 3; ++j) h.a[j] = draw64(key, (uint64_t)j) % kP31;
  for (int j = 0; j < 4; ++j) h.b[j] = draw64(key, (uint64_t)(3 + j)) % kP31;
  return h;
}

// Horner evaluation mod p; every intermediate stays below 2^62 + 2^31.
__device__ __forceinline__ uint64_t poly_mod_p(const uint64_t* c, int ncoef, uint64_t x) {
  uint64_t acc = c[ncoef - 1];
  for (int j = ncoef - 2; j >= 0; --j) acc = (acc * x + c[j]) % kP31;
  return acc;
}

__device__ __forceinline__ int32_t pack_entry(uint32_t bin, bool negative) {
  return (int32_t)(bin | (negative ? 0x80000000u : 0u));
}
__device__ __forceinline__ int entry_bin(int32_t p) { return p & 0x7fffffff; }
__device__ __forceinline__ bool entry_neg(int32_t p) { return p < 0; }

// ---------------------------------------------------------------- complex

template <typename T>
struct Cx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ Cx<T> cadd(Cx<T> a, Cx<T> b) {
  return {a.x + b.x, a.y + b.y};
}
template <typename T>
__device__ __forceinline__ Cx<T> csub(Cx<T> a, Cx<T> b) {
  return {a.x - b.x, a.y - b.y};
}
template <typename T>
__device__ __forceinline__ Cx<T> cconj(Cx<T> a) {
  return {a.x, -a.y};
}

// ---------------------------------------------------------------- dtype helpers

inline size_t dtype_size(int dt) { return dt == TS_F64 ? 8 : 4; }

}  // namespace ts
