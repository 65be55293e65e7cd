// rt_peaks.cu -- FMA-throughput microbenchmark (measurement support; the
// paper has no counterpart). Every thread runs independent FMA chains
// x <- x * a + b long enough to hide the pipe latency; the grid fills every
// SM several times over. FLOPs = 2 per FMA.
#include <cuda_runtime.h>

#include "../../include/rt_cnop.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_chains(int iters, T a, T b, T* out) {
  T x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) x[k] = fma(x[k], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains alive
}

template <class T>
cudaError_t time_fma(int blocks, int iters, double* tflops) {
  T* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t err = cudaMalloc(&out, (size_t)blocks * kThreads * sizeof(T));
  if (err == cudaSuccess) err = cudaEventCreate(&e0);
  if (err == cudaSuccess) err = cudaEventCreate(&e1);
  float best = 0.f;
  for (int rep = 0; err == cudaSuccess && rep < 4; ++rep) {  // rep 0 warms up
    cudaEventRecord(e0);
    k_fma_chains<T><<<blocks, kThreads>>>(iters, T(0.999999), T(1e-6), out);
    cudaEventRecord(e1);
    err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (err == cudaSuccess && best > 0.f)
    *tflops = 2.0 * kChains * (double)iters * blocks * kThreads / (best * 1e-3) / 1e12;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  return err;
}

}  // namespace

extern "C" rt_status rt_fma_peak(double* tflops_f32, double* tflops_f64) {
  if (!tflops_f32 || !tflops_f64) return RT_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
    return RT_ECUDA;
  *tflops_f32 = *tflops_f64 = 0.0;
  if (time_fma<float>(sms * 16, 4096, tflops_f32) != cudaSuccess) return RT_ECUDA;
  if (time_fma<double>(sms * 16, 256, tflops_f64) != cudaSuccess) return RT_ECUDA;
  return RT_OK;
}
