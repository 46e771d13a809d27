// One-pass sketch of the data tensor (Alg. 4, right-hand side): for every stored
// entry (i, v) and every requested output ("job") with mode n and bucket count M,
//   Y_n[(sum_{k != n} H_{n,k}(i_k)) mod M, i_n] += prod_{k != n} S_{n,k}(i_k) v.
// Several outputs share a single read of the tensor.  Used for the TensorSketch
// right-hand sides (M = m) and for the CountSketch factor of Init-RRF (M = k2).
#include "internal.cuh"

namespace ts {

struct JobsDesc {
  int njobs;
  int order;
  int64_t dims[TS_MAX_ORDER];
  int mode[kMaxJobs];
  int nbins[kMaxJobs];
  void* out[kMaxJobs];
  const int32_t* tab[kMaxJobs][TS_MAX_ORDER];
};

template <typename T>
__device__ __forceinline__ void scatter_entry(const JobsDesc& d, const int64_t* idx, T v) {
  for (int j = 0; j < d.njobs; ++j) {
    const int n = d.mode[j];
    int64_t bin = 0;
    bool neg = false;
    for (int k = 0; k < d.order; ++k) {
      if (k == n) continue;
      const int32_t e = __ldg(d.tab[j][k] + idx[k]);
      bin += entry_bin(e);
      neg ^= entry_neg(e);
    }
    bin %= d.nbins[j];
    T* Y = static_cast<T*>(d.out[j]);
    atomicAdd(Y + bin * d.dims[n] + idx[n], neg ? -v : v);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_sketch_dense_generic(JobsDesc d, const T* __restrict__ X,
                                                              int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t idx[TS_MAX_ORDER];
    int64_t r = e;
    for (int k = d.order - 1; k >= 0; --k) {
      idx[k] = r % d.dims[k];
      r /= d.dims[k];
    }
    scatter_entry<T>(d, idx, X[e]);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_sketch_coo(JobsDesc d, const int32_t* __restrict__ I,
                                                    const T* __restrict__ V, int64_t nnz) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t idx[TS_MAX_ORDER];
    bool ok = true;
    for (int k = 0; k < d.order; ++k) {
      idx[k] = I[k * nnz + e];
      ok &= (idx[k] >= 0) & (idx[k] < d.dims[k]);
    }
    if (ok) scatter_entry<T>(d, idx, V[e]);  // out-of-range coordinates are skipped
  }
}

template <typename T>
ts_status launch_input_sketch(const ts_tensor& X, const SketchJob* jobs, int njobs, int* flag,
                              cudaStream_t st) {
  if (njobs < 1) return TS_OK;
  if (njobs > kMaxJobs) return fail(TS_ERR_INVALID_ARG, "input sketch: too many outputs");
  if (sizeof(T) == 4 && dense3_tma_eligible(X, jobs, njobs) &&
      dense3_tma_smem_bytes(X, jobs, njobs) <= kMaxSmem)
    return launch_dense3_tma(X, jobs, njobs, flag, st);
  JobsDesc d{};
  d.njobs = njobs;
  d.order = X.order;
  for (int k = 0; k < X.order; ++k) d.dims[k] = X.dims[k];
  for (int j = 0; j < njobs; ++j) {
    d.mode[j] = jobs[j].mode;
    d.nbins[j] = jobs[j].nbins;
    d.out[j] = jobs[j].out;
    for (int k = 0; k < X.order; ++k) d.tab[j][k] = jobs[j].tables[k];
    TS_CUDA(cudaMemsetAsync(jobs[j].out, 0,
                            sizeof(T) * (size_t)jobs[j].nbins * (size_t)X.dims[jobs[j].mode], st));
  }
  if (X.format == TS_DENSE) {
    int64_t total = 1;
    for (int k = 0; k < X.order; ++k) total *= X.dims[k];
    long blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_sketch_dense_generic<T><<<(int)blocks, 256, 0, st>>>(d, static_cast<const T*>(X.values),
                                                           total);
  } else {
    if (X.nnz == 0) return TS_OK;
    long blocks = (X.nnz + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_sketch_coo<T><<<(int)blocks, 256, 0, st>>>(d, X.indices, static_cast<const T*>(X.values),
                                                 X.nnz);
  }
  TS_LAUNCH_CHECK();
  return TS_OK;
}

template ts_status launch_input_sketch<float>(const ts_tensor&, const SketchJob*, int, int*,
                                              cudaStream_t);
template ts_status launch_input_sketch<double>(const ts_tensor&, const SketchJob*, int, int*,
                                               cudaStream_t);

}  // namespace ts
