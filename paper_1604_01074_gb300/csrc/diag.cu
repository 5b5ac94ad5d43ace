// Diagnostics without a counterpart in the paper: the fused multiply-add throughput of
// the GPU in float64 or float32, the ceiling of a solve that is bound by arithmetic
// rather than by memory (float64 packs: 2 flops per matrix entry against 1/64 of the
// float32 rate on this GPU).
//
// Each thread runs 8 independent FMA chains (enough to cover the pipeline latency) for
// `iters` steps; 8 CTAs of 256 threads per SM.  The chains' sums are written out so the
// arithmetic cannot be dropped.  Timed with CUDA events around one launch after a
// warm-up launch.
#include <cuda_runtime.h>

#include "smpc_internal.h"

namespace smpc {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_chains(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
int run_peak(double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    set_error("no CUDA device");
    return SMPC_ECUDA;
  }
  const int grid = 8 * sms, block = 256;
  const int iters = sizeof(T) == 8 ? 4096 : 65536;
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * (size_t)grid * block) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc failed");
    return SMPC_ENOMEM;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = SMPC_OK;
  float ms = 0;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = SMPC_ECUDA;
  if (rc == SMPC_OK) {
    // a = 1 - 2^-20, b = 2^-20: the chains stay bounded near 1
    const T a = (T)(1.0 - 1.0 / 1048576.0), b = (T)(1.0 / 1048576.0);
    fma_chains<T><<<grid, block>>>(out, iters / 8, a, b);  // warm-up
    cudaEventRecord(e0);
    fma_chains<T><<<grid, block>>>(out, iters, a, b);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0) {
      set_error("FMA timing failed: %s", cudaGetErrorString(cudaGetLastError()));
      rc = SMPC_ECUDA;
    }
  }
  if (rc == SMPC_OK) *tflops = 2.0 * 8.0 * iters * (double)grid * block / (ms * 1e-3) / 1e12;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return rc;
}

}  // namespace
}  // namespace smpc

extern "C" int smpc_fma_peak(int32_t precision, double* tflops) {
  if (!tflops || (precision != SMPC_FP64 && precision != SMPC_FP32)) {
    smpc::set_error("smpc_fma_peak: precision SMPC_FP64 or SMPC_FP32 and a result pointer");
    return SMPC_EINVAL;
  }
  return precision == SMPC_FP64 ? smpc::run_peak<double>(tflops) : smpc::run_peak<float>(tflops);
}
