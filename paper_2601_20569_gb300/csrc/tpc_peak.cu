// Arithmetic peaks of the device the library runs on, measured: FP32 and FP64
// fused multiply-add throughput of a kernel that does nothing else (eight
// independent FMA chains per thread, no memory traffic but one store per
// thread at the end).  The fit kernels' ncu pipe utilisation is read against
// these numbers; the paper has no counterpart.
#include <cuda_runtime.h>

#include "tpc.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_fma_peak(T a, T b, int iters, T* out) {
  T v[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) v[j] = T(threadIdx.x + j) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int j = 0; j < kChains; ++j) v[j] = fma(v[j], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += v[j];
  out[(long)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
tpc_status time_peak(int iters, double* tflops, cudaStream_t s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TPC_ERR_CUDA;
  const int blocks = sms * 8;
  T* out = nullptr;
  if (cudaMallocAsync((void**)&out, sizeof(T) * blocks * kThreads, s) != cudaSuccess)
    return TPC_ERR_OOM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  tpc_status st = TPC_OK;
  float ms = 0.0f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = TPC_ERR_CUDA;
  } else {
    // a multiplier just below 1 and a small addend keep the chains finite
    k_fma_peak<T><<<blocks, kThreads, 0, s>>>(T(0.999999), T(1e-6), iters / 8 + 1, out);  // warm
    cudaEventRecord(e0, s);
    k_fma_peak<T><<<blocks, kThreads, 0, s>>>(T(0.999999), T(1e-6), iters, out);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        cudaGetLastError() != cudaSuccess)
      st = TPC_ERR_CUDA;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(out, s);
  if (st == TPC_OK) {
    const double flops = 2.0 * kChains * 16.0 * iters * (double)blocks * kThreads;
    *tflops = ms > 0.0f ? flops / (ms * 1e-3) / 1e12 : 0.0;
  }
  return st;
}

}  // namespace

extern "C" tpc_status tpc_fma_peak(int32_t fp64, int32_t iters, double* tflops,
                                   void* cuda_stream) {
  if (!tflops || iters < 1) return TPC_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  return fp64 ? time_peak<double>(iters, tflops, s) : time_peak<float>(iters, tflops, s);
}
