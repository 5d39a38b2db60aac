// Measured FMA throughput (include/hfx_peak.h): 8 independent dependency chains per thread, enough
// resident blocks to fill every SM, CUDA events around the launch.
#include <cuda_runtime.h>

#include "../../include/hfx_peak.h"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) k_fma_chains(T* out, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = T(threadIdx.x + j) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = fma(x[j], a, b);
  }
  T s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
hfx_status run(int iters, double* tflops, cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HFX_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HFX_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_chains<T>, 256, 0) != cudaSuccess) return HFX_ERR_CUDA;
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  T* out = nullptr;
  if (cudaMalloc(&out, sizeof(T) * (size_t)grid * 256) != cudaSuccess) return HFX_ERR_CUDA;
  cudaEvent_t a = nullptr, b = nullptr;
  hfx_status status = HFX_OK;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) status = HFX_ERR_CUDA;
  if (status == HFX_OK) {
    k_fma_chains<T><<<grid, 256, 0, st>>>(out, iters / 10 + 1, T(0.999999), T(1e-7));  // warm-up
    cudaEventRecord(a, st);
    k_fma_chains<T><<<grid, 256, 0, st>>>(out, iters, T(0.999999), T(1e-7));
    cudaEventRecord(b, st);
    float ms = 0.f;
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
        cudaEventElapsedTime(&ms, a, b) != cudaSuccess || ms <= 0.f)
      status = HFX_ERR_CUDA;
    else
      *tflops = 2.0 * 8.0 * (double)iters * (double)grid * 256.0 / (ms * 1e-3) / 1e12;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(out);
  return status;
}

}  // namespace

extern "C" hfx_status hfx_fma_peak(int32_t fp64, int32_t iters, double* tflops, void* cuda_stream) {
  if (iters < 1 || !tflops) return HFX_ERR_INVALID_ARG;
  return fp64 ? run<double>(iters, tflops, (cudaStream_t)cuda_stream)
              : run<float>(iters, tflops, (cudaStream_t)cuda_stream);
}
