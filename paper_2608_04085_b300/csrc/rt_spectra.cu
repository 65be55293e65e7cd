// rt_spectra.cu -- Fourier analysis of perturbation fields (Sec. 4.2
// Eq. fourier_coeff, Sec. 3.5, App. B). See rt_spectra.h.
//
// The transforms are plain DFTs: one CTA per row (or column) stages the data
// and the n twiddles exp(sign 2 pi i m / n), m = 0 .. n-1, in shared memory,
// and output k accumulates in[j] * twiddle[(k j) mod n] with the index
// advanced by k modulo n, so every phase is reduced exactly. The fields are at
// most a few million values and the analysis runs once per CNOP, so the
// O(n) work per output is not worth an FFT here.
#include "rt_spectra.h"

namespace rt {
namespace {

constexpr int NTH_DFT = 256;
constexpr int NTH_ONE = 1024;  // single-CTA selection kernels

__global__ void __launch_bounds__(NTH_DFT) k_dft_x(const double2* __restrict__ in, double2* __restrict__ out, int nx,
                                                   double sign) {
  extern __shared__ double2 sm[];
  double2* row = sm;
  double2* tw = sm + nx;
  const long long base = (long long)blockIdx.x * nx;
  for (int j = threadIdx.x; j < nx; j += blockDim.x) {
    row[j] = in[base + j];
    double sn, cs;
    sincospi(2.0 * j / nx, &sn, &cs);
    tw[j] = make_double2(cs, sign * sn);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nx; k += blockDim.x) {
    double re = 0.0, im = 0.0;
    int m = 0;
    for (int j = 0; j < nx; ++j) {
      const double2 a = row[j], t = tw[m];
      re += a.x * t.x - a.y * t.y;
      im += a.x * t.y + a.y * t.x;
      m += k;
      if (m >= nx) m -= nx;
    }
    out[base + k] = make_double2(re, im);
  }
}

__global__ void __launch_bounds__(NTH_DFT) k_dft_y(const double2* __restrict__ in, double2* __restrict__ out, int nx,
                                                   int ny, double sign) {
  extern __shared__ double2 sm[];
  double2* col = sm;
  double2* tw = sm + ny;
  const int x = blockIdx.x;
  for (int l = threadIdx.x; l < ny; l += blockDim.x) {
    col[l] = in[(long long)l * nx + x];
    double sn, cs;
    sincospi(2.0 * l / ny, &sn, &cs);
    tw[l] = make_double2(cs, sign * sn);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < ny; k += blockDim.x) {
    double re = 0.0, im = 0.0;
    int m = 0;
    for (int l = 0; l < ny; ++l) {
      const double2 a = col[l], t = tw[m];
      re += a.x * t.x - a.y * t.y;
      im += a.x * t.y + a.y * t.x;
      m += k;
      if (m >= ny) m -= ny;
    }
    out[(long long)k * nx + x] = make_double2(re, im);
  }
}

__global__ void k_real_to_complex(const double* __restrict__ f, double2* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = make_double2(f[i], 0.0);
}

__global__ void k_real_part(const double2* __restrict__ in, double* __restrict__ out, long long n, double scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = scale * in[i].x;
}

__global__ void k_power(const double2* __restrict__ F, double* __restrict__ E, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    E[i] = F[i].x * F[i].x + F[i].y * F[i].y;
}

__global__ void k_mask(double2* __restrict__ F, const unsigned char* __restrict__ keep, int nx, long long n, int mode) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const bool k = mode == 0 ? keep[i % nx] != 0 : keep[i] != 0;
    if (!k) F[i] = make_double2(0.0, 0.0);
  }
}

// Sum (or max, for non-negative values) over the block, returned to every thread.
template <bool MAX>
__device__ double block_all(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = MAX ? fmax(v, w) : v + w;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = MAX ? fmax(s, red[w]) : s + red[w];
    red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// Energy of the conjugate pair {k, -k} of mode k; rep: k is the pair's representative.
__device__ __forceinline__ double pair_energy(const double* E, long long k, int nx, int ny, bool& rep) {
  const int ky = (int)(k / nx), kx = (int)(k % nx);
  const long long c = (long long)((ny - ky) % ny) * nx + (nx - kx) % nx;
  rep = k <= c;
  return c == k ? E[k] : E[k] + E[c];
}

__global__ void __launch_bounds__(NTH_ONE) k_select_pairs(const double* __restrict__ E, int nx, int ny, double frac,
                                                          unsigned char* __restrict__ keep, int* __restrict__ kept,
                                                          double* __restrict__ total) {
  __shared__ double red[33];
  const long long n = (long long)nx * ny;
  auto kept_sum = [&](double tau) {
    double s = 0.0;
    for (long long k = threadIdx.x; k < n; k += blockDim.x) {
      bool rep;
      const double p = pair_energy(E, k, nx, ny, rep);
      if (rep && p >= tau) s += p;
    }
    return block_all<false>(s, red);
  };
  double mx = 0.0;
  for (long long k = threadIdx.x; k < n; k += blockDim.x) {
    bool rep;
    mx = fmax(mx, pair_energy(E, k, nx, ny, rep));
  }
  mx = block_all<true>(mx, red);
  const double T = kept_sum(0.0);
  // largest threshold (as ordered bit patterns of non-negative doubles) whose
  // kept pairs still hold frac of the energy
  unsigned long long lo = 0, hi = (unsigned long long)__double_as_longlong(mx) + 1ull;
  while (hi - lo > 1ull) {
    const unsigned long long mid = lo + (hi - lo) / 2ull;
    if (kept_sum(__longlong_as_double((long long)mid)) >= frac * T) lo = mid;
    else hi = mid;
  }
  const double tau = __longlong_as_double((long long)lo);
  double cnt = 0.0;
  for (long long k = threadIdx.x; k < n; k += blockDim.x) {
    bool rep;
    const bool in = pair_energy(E, k, nx, ny, rep) >= tau;
    keep[k] = in ? 1 : 0;
    cnt += in ? 1.0 : 0.0;
  }
  cnt = block_all<false>(cnt, red);
  if (threadIdx.x == 0) {
    *kept = (int)cnt;
    *total = T;
  }
}

__global__ void __launch_bounds__(NTH_ONE) k_rms_peak(const double* __restrict__ f, int nx, int ny,
                                                      int* __restrict__ y_peak) {
  __shared__ double bv[NTH_ONE];
  __shared__ int bi[NTH_ONE];
  double best = -1.0;
  int at = 0;  // stays in range even for a field of NaNs
  for (int y = threadIdx.x; y < ny; y += blockDim.x) {
    double s = 0.0;
    for (int x = 0; x < nx; ++x) s += f[(long long)y * nx + x] * f[(long long)y * nx + x];
    const double r = sqrt(s / nx);
    if (r > best) {  // rows visited in increasing order: ties keep the lower row
      best = r;
      at = y;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = at;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double v2 = bv[threadIdx.x + o];
      const int i2 = bi[threadIdx.x + o];
      if (v2 > bv[threadIdx.x] || (v2 == bv[threadIdx.x] && i2 < bi[threadIdx.x])) {
        bv[threadIdx.x] = v2;
        bi[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *y_peak = bi[0];
}

__global__ void __launch_bounds__(NTH_ONE) k_select_x(const double2* __restrict__ X, int nx,
                                                      const int* __restrict__ y_peak, int count,
                                                      double* __restrict__ E, unsigned char* __restrict__ keepx,
                                                      int* __restrict__ kept) {
  __shared__ double red[33];
  const int half = nx / 2;
  const double2* row = X + (long long)(*y_peak) * nx;
  double s = 0.0;
  for (int n = 1 + threadIdx.x; n <= half; n += blockDim.x) {
    const double p = row[n].x * row[n].x + row[n].y * row[n].y;
    E[n - 1] = p;
    s += p;
  }
  for (int k = threadIdx.x; k < nx; k += blockDim.x) keepx[k] = 0;
  s = block_all<false>(s, red);
  for (int n = 1 + threadIdx.x; n <= half; n += blockDim.x) E[n - 1] = E[n - 1] / s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int k = 0;
    for (int r = 0; r < count && r < half; ++r) {
      int at = -1;
      for (int n = 1; n <= half; ++n)  // first maximum: ties keep the lower n
        if (!keepx[n] && (at < 0 || E[n - 1] > E[at - 1])) at = n;
      keepx[at] = 1;
      keepx[(nx - at) % nx] = 1;
      k += at == (nx - at) % nx ? 1 : 2;  // modes kept: n and its mirror -n
    }
    *kept = k;
  }
}

__global__ void k_scale_by(double* __restrict__ E, long long n, const double* __restrict__ denom) {
  const double d = *denom;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    E[i] = E[i] / d;
}

int grid_for(long long n) {
  const long long b = (n + 255) / 256;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

cudaError_t spec_configure() {
  const int bytes = 2 * SPEC_MAX_N * (int)sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(k_dft_x, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_dft_y, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

cudaError_t spec_dft_x(const double2* in, double2* out, int nx, int ny, double sign, cudaStream_t s) {
  k_dft_x<<<ny, NTH_DFT, 2 * nx * sizeof(double2), s>>>(in, out, nx, sign);
  return cudaGetLastError();
}

cudaError_t spec_dft_y(const double2* in, double2* out, int nx, int ny, double sign, cudaStream_t s) {
  k_dft_y<<<nx, NTH_DFT, 2 * ny * sizeof(double2), s>>>(in, out, nx, ny, sign);
  return cudaGetLastError();
}

cudaError_t spec_real_to_complex(const double* f, double2* out, long long n, cudaStream_t s) {
  k_real_to_complex<<<grid_for(n), 256, 0, s>>>(f, out, n);
  return cudaGetLastError();
}

cudaError_t spec_real_part(const double2* in, double* out, long long n, double scale, cudaStream_t s) {
  k_real_part<<<grid_for(n), 256, 0, s>>>(in, out, n, scale);
  return cudaGetLastError();
}

cudaError_t spec_power(const double2* F, double* E, long long n, cudaStream_t s) {
  k_power<<<grid_for(n), 256, 0, s>>>(F, E, n);
  return cudaGetLastError();
}

cudaError_t spec_select_pairs(const double* E, int nx, int ny, double frac, unsigned char* keep, int* kept,
                              double* total, cudaStream_t s) {
  k_select_pairs<<<1, NTH_ONE, 0, s>>>(E, nx, ny, frac, keep, kept, total);
  return cudaGetLastError();
}

cudaError_t spec_rms_peak(const double* f, int nx, int ny, int* y_peak, cudaStream_t s) {
  k_rms_peak<<<1, NTH_ONE, 0, s>>>(f, nx, ny, y_peak);
  return cudaGetLastError();
}

cudaError_t spec_select_x(const double2* X, int nx, const int* y_peak, int count, double* E, unsigned char* keepx,
                          int* kept, cudaStream_t s) {
  k_select_x<<<1, NTH_ONE, 0, s>>>(X, nx, y_peak, count, E, keepx, kept);
  return cudaGetLastError();
}

cudaError_t spec_scale_by(double* E, long long n, const double* denom, cudaStream_t s) {
  k_scale_by<<<grid_for(n), 256, 0, s>>>(E, n, denom);
  return cudaGetLastError();
}

cudaError_t spec_mask(double2* F, const unsigned char* keep, int nx, int ny, int mode, cudaStream_t s) {
  const long long n = (long long)nx * ny;
  k_mask<<<grid_for(n), 256, 0, s>>>(F, keep, nx, n, mode);
  return cudaGetLastError();
}

}  // namespace rt
