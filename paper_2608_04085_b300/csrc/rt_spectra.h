// rt_spectra.h -- device side of the Fourier analysis of perturbation fields
// (Sec. 4.2 Eq. fourier_coeff, Sec. 3.5, App. B). Plain DFTs with exactly
// reduced phases, spectral energies and the mode selections of the five-mode
// and the power-fraction reconstructions. FP64, off the time-stepping path.
// Fields are one instance's [ny][nx] planes, row-major, x fastest.
#pragma once
#include <cuda_runtime.h>

namespace rt {

// Largest transform length a DFT kernel accepts (row or column staged in
// shared memory with its twiddles).
constexpr int SPEC_MAX_N = 6144;

cudaError_t spec_configure();
// out[y][k] = sum_j in[y][j] exp(sign 2 pi i k j / nx), every row
cudaError_t spec_dft_x(const double2* in, double2* out, int nx, int ny, double sign, cudaStream_t s);
// out[k][x] = sum_l in[l][x] exp(sign 2 pi i k l / ny), every column
cudaError_t spec_dft_y(const double2* in, double2* out, int nx, int ny, double sign, cudaStream_t s);
cudaError_t spec_real_to_complex(const double* f, double2* out, long long n, cudaStream_t s);
// out = scale * Re(in)
cudaError_t spec_real_part(const double2* in, double* out, long long n, double scale, cudaStream_t s);
cudaError_t spec_power(const double2* F, double* E, long long n, cudaStream_t s);
// keep[k] = 1 for the conjugate mode pairs holding `frac` of sum E (largest
// pairs first, ties with the last kept pair included); kept = modes kept,
// total = sum E. One CTA.
cudaError_t spec_select_pairs(const double* E, int nx, int ny, double frac, unsigned char* keep, int* kept,
                              double* total, cudaStream_t s);
// y_peak = row of the largest rms of f (ties: lowest row). One CTA.
cudaError_t spec_rms_peak(const double* f, int nx, int ny, int* y_peak, cudaStream_t s);
// From the row DFT X of the field: E[n - 1] = |X[y_peak][n]|^2 normalised over
// n = 1 .. nx/2, and keepx[] marking the `count` largest n (ties: lower n)
// with their mirrors nx - n. One CTA.
cudaError_t spec_select_x(const double2* X, int nx, const int* y_peak, int count, double* E, unsigned char* keepx,
                          int* kept, cudaStream_t s);
// E[i] /= *denom for i < n
cudaError_t spec_scale_by(double* E, long long n, const double* denom, cudaStream_t s);
// zero the modes not kept: mode 0 keep[kx] (every row), mode 1 keep[ky*nx+kx]
cudaError_t spec_mask(double2* F, const unsigned char* keep, int nx, int ny, int mode, cudaStream_t s);

}  // namespace rt
