// rt_kernels_f64.cu -- FP64 instantiation of the kernels, plus the FP64
// field kernels. Compiled with -fmad=false: every product and sum rounds on
// its own, exactly as the scheme's expressions are written.
#define RT_FIELD_KERNELS 1
#include "rt_launch_impl.cuh"

namespace rt {
RT_INSTANTIATE_LAUNCHERS(double)

cudaError_t launch_finalize(const InstDev* insts, int n_inst, const double* partials, int width, int scale_by_dA,
                            double* out, cudaStream_t s) {
  k_finalize<<<n_inst, NTH, 0, s>>>(insts, partials, width, scale_by_dA, out);
  return cudaGetLastError();
}

cudaError_t launch_field_reduce(int mode, const InstDev* insts, const int4* tiles, int ntiles, const double* a,
                                const double* b, double* partials, cudaStream_t s) {
  if (mode == 0) k_field_reduce<0><<<ntiles, NTH, 0, s>>>(insts, tiles, a, b, partials);
  else if (mode == 1) k_field_reduce<1><<<ntiles, NTH, 0, s>>>(insts, tiles, a, b, partials);
  else k_field_reduce<2><<<ntiles, NTH, 0, s>>>(insts, tiles, a, b, partials);
  return cudaGetLastError();
}

cudaError_t launch_series_sample(const InstDev* insts, int n_inst, const double2* rowsum, const double* t,
                                 const int* nstep, double* out, cudaStream_t s) {
  k_series_sample<<<n_inst, NTH, 0, s>>>(insts, rowsum, t, nstep, out);
  return cudaGetLastError();
}

cudaError_t launch_dt_coef(const InstDev* insts, int n_inst, const double* partials, const RunDev& run, int n,
                           double* blast, double* coef, cudaStream_t s) {
  k_dt_coef<<<n_inst, NTH, 0, s>>>(insts, partials, run, n, blast, coef);
  return cudaGetLastError();
}

cudaError_t launch_finalize_max(const InstDev* insts, int n_inst, const double* partials, double* out,
                                cudaStream_t s) {
  k_finalize_max<<<n_inst, NTH, 0, s>>>(insts, partials, out);
  return cudaGetLastError();
}

cudaError_t launch_field_axpby(const InstDev* insts, const int4* tiles, int ntiles, double* out,
                               const double* alpha, const double* a, const double* beta, const double* b,
                               cudaStream_t s) {
  k_field_axpby<<<ntiles, NTH, 0, s>>>(insts, tiles, out, alpha, a, beta, b);
  return cudaGetLastError();
}

cudaError_t launch_field_weight(const InstDev* insts, const int4* tiles, int ntiles, double* out, const double* a,
                                int inverse, cudaStream_t s) {
  k_field_weight<<<ntiles, NTH, 0, s>>>(insts, tiles, out, a, inverse);
  return cudaGetLastError();
}

cudaError_t launch_localise(const InstDev* insts, const int4* tiles, int ntiles, double h_loc, double* v,
                            cudaStream_t s) {
  k_localise<<<ntiles, NTH, 0, s>>>(insts, tiles, h_loc, v);
  return cudaGetLastError();
}
}  // namespace rt
