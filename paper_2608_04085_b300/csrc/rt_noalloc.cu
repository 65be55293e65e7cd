// rt_noalloc.cu -- allocation-free objective evaluation (rt_objective_noalloc).
//
// Some callers cannot let a library allocate device memory: code that runs
// under a host framework which owns every device byte through its own pool or
// arena with a fixed budget, or a latency-critical loop that cannot afford
// the device-wide synchronisation that cudaMalloc/cudaFree imply. For them
// this file offers one entry point that evaluates the objective of a final
// state (the sums the forward run ends with) without any allocation: the
// caller passes the state and the output, and the per-block partial sums live
// in a fixed file-scope device array.
//
// That array (kMaxBlocks * 2 doubles = 256 KiB) is part of the library image:
// every GPU on which the library is loaded holds it until the process exits.
// It bounds the problem size at kMaxCells = 4,194,304 cells; larger grids are
// rejected with RT_EINVAL. All calls share it: two calls whose kernels overlap
// on the GPU (different streams, or different host threads) race on it and
// may return wrong sums. Each call writes every partial it later reads, so no
// part of the array has to start at zero and stale contents from an earlier
// call are never read.
#include <cstdio>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/rt_cnop.h"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 16384;
constexpr long long kMaxCells = (long long)kMaxBlocks * kThreads;
constexpr int kMaxDevices = 64;

// Per-block partial sums: [2*b] = sum of e_k, [2*b+1] = sum of (e_k - e_k0)^2.
static __device__ __align__(256) double g_partials[2 * kMaxBlocks];

// Device address of g_partials, looked up once per device. In host code the
// symbol's name is only a host-side stand-in, so kernels get this address.
// The cache lives as long as the process; a cudaDeviceReset unloads the
// device image it points into, so calls after a reset are not supported.
double* g_addr[kMaxDevices] = {nullptr};
std::mutex g_mu;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// e_k = rho |u|^2 / 2 of each cell and its block sums (fixed order).
__global__ void __launch_bounds__(kThreads) k_ek_partials(const double* __restrict__ U, const double* __restrict__ ek0,
                                                          long long cells, double* __restrict__ partials) {
  __shared__ double red[2][kThreads / 32];
  const long long c = (long long)blockIdx.x * kThreads + threadIdx.x;
  double ke = 0.0, pap = 0.0;
  if (c < cells) {
    const double r = U[c], mx = U[cells + c], my = U[2 * cells + c];
    const double ek = 0.5 * (mx * mx + my * my) / r;
    const double a = ek - (ek0 ? ek0[c] : 0.0);
    ke = ek;
    pap = a * a;
  }
  ke = warp_sum(ke);
  pap = warp_sum(pap);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = ke;
    red[1][wid] = pap;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    partials[2 * blockIdx.x] = s0;
    partials[2 * blockIdx.x + 1] = s1;
  }
}

// J[0] = dA * sum e_k, J[1] = dA * sum (e_k - e_k0)^2 over the nblocks partials.
__global__ void __launch_bounds__(kThreads) k_ek_sum(const double* __restrict__ partials, int nblocks, double dA,
                                                     double* __restrict__ J) {
  __shared__ double red[2][kThreads / 32];
  double s0 = 0.0, s1 = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += kThreads) {
    s0 += partials[2 * b];
    s1 += partials[2 * b + 1];
  }
  s0 = warp_sum(s0);
  s1 = warp_sum(s1);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = s0;
    red[1][wid] = s1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0.0, t1 = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) {
      t0 += red[0][w];
      t1 += red[1][w];
    }
    J[0] = t0 * dA;
    J[1] = t1 * dA;
  }
}

// Set-up, once per device, with that device current: the device address of
// the scratch array. Returns null (and prints why) if the lookup fails.
double* scratch_for_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    fprintf(stderr, "rt_objective_noalloc: no usable current CUDA device\n");
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
    if (e != cudaSuccess) {
      fprintf(stderr, "rt_objective_noalloc: cudaGetSymbolAddress failed on device %d: %s\n", dev,
              cudaGetErrorString(e));
      return nullptr;
    }
    g_addr[dev] = static_cast<double*>(p);
  }
  return g_addr[dev];
}

}  // namespace

extern "C" rt_status rt_objective_noalloc(const rt_problem* p, const double* state, const double* ek0, double* J,
                                          void* cuda_stream) {
  if (!p || !state || !J) {
    fprintf(stderr, "rt_objective_noalloc: null argument\n");
    return RT_EINVAL;
  }
  const long long cells = (long long)p->nx * p->ny;
  if (p->nx <= 0 || p->ny <= 0 || cells > kMaxCells) {
    fprintf(stderr, "rt_objective_noalloc: grid %d x %d outside 1 .. %lld cells (fixed scratch limit)\n", p->nx,
            p->ny, kMaxCells);
    return RT_EINVAL;
  }
  if (!(p->x1 > p->x0) || !(p->y1 > p->y0)) {
    fprintf(stderr, "rt_objective_noalloc: empty domain\n");
    return RT_EINVAL;
  }
  double* scratch = scratch_for_current_device();
  if (!scratch) return RT_ECUDA;
  const double dA = ((p->x1 - p->x0) / p->nx) * ((p->y1 - p->y0) / p->ny);
  const int nblocks = (int)((cells + kThreads - 1) / kThreads);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  k_ek_partials<<<nblocks, kThreads, 0, s>>>(state, ek0, cells, scratch);
  k_ek_sum<<<1, kThreads, 0, s>>>(scratch, nblocks, dA, J);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    fprintf(stderr, "rt_objective_noalloc: launch failed: %s\n", cudaGetErrorString(e));
    return RT_ECUDA;
  }
  return RT_OK;
}
