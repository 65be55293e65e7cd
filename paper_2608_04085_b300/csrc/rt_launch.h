// rt_launch.h -- host-side launchers of the kernels (defined in the FP32 and
// FP64 translation units) used by the runtime.
#pragma once

#include <cuda_runtime.h>

#include "rt_internal.h"

namespace rt {

template <class T>
cudaError_t launch_inject(const InstDev* insts, const int4* tiles, int ntiles, const double* v, T* U,
                          const RunDev& run, int record, cudaStream_t s);
// variant: STAGE_SWEEP or a tile variant; mode: 0 CFL control, 1 replay
// counting steps, 2 replay (recompute)
// lim: the batch's common limiter (compile-time specialised kernels), or -1
// tm: TMA maps of src (tile variants; boxes of tile height + 4 rows)
template <class T>
cudaError_t launch_stage(int variant, int lim, int stage, int mode, const InstDev* insts, const int4* strips,
                         int nstrips, const int4* tiles, int ntiles, const T* src, const T* base, T* dst,
                         const RunDev& run, int n, const TileMaps& tm, cudaStream_t s);
// rows: the adjoint tile height (16, or 24 for FP32) of the work list
// `tiles`; tmu, tmk: TMA maps of U (boxes of rows + 6 rows) and K (rows + 4)
template <class T>
cudaError_t launch_adjoint(int rows, int lim, const InstDev* insts, const int4* tiles, int ntiles, const T* U,
                           const T* K, double kscale, const T* E, double escale, T* out, const RunDev& run, int n,
                           const TileMaps& tmu, const TileMaps& tmk, cudaStream_t s);
template <class T>
cudaError_t launch_objective(const InstDev* insts, const int4* tiles, int ntiles, T* const* slot_tab, int tab_mod,
                             const int* nstep, double* ek_out, T* lamA, T* lamB, double* partials,
                             cudaStream_t s);
template <class T>
cudaError_t launch_row_sums(const InstDev* insts, const int2* rows, int nrows, T* const* slot_tab, const int* nstep,
                            double2* out, cudaStream_t s);
// one diagnostics sample per instance: out[i] = {t, KE, h_mix, nstep}
cudaError_t launch_series_sample(const InstDev* insts, int n_inst, const double2* rowsum, const double* t,
                                 const int* nstep, double* out, cudaStream_t s);
// gradient through the step control (see k_dt_partials / k_dt_coef / k_dt_apply)
template <class T>
cudaError_t launch_dt_partials(const InstDev* insts, const int4* tiles, int ntiles, const T* U, const T* U1,
                               const T* Un1, const T* lam, const T* lam1, const RunDev& run, int n, double* partials,
                               cudaStream_t s);
cudaError_t launch_dt_coef(const InstDev* insts, int n_inst, const double* partials, const RunDev& run, int n,
                           double* blast, double* coef, cudaStream_t s);
template <class T>
cudaError_t launch_dt_apply(const InstDev* insts, const int4* tiles, int ntiles, const T* U, T* lam, const RunDev& run,
                            int n, const double* coef, cudaStream_t s);
template <class T>
cudaError_t launch_grad(const InstDev* insts, const int4* tiles, int ntiles, const T* lam, const double* v,
                        double* g, cudaStream_t s);
template <class T>
cudaError_t configure_kernels();

cudaError_t launch_finalize(const InstDev* insts, int n_inst, const double* partials, int width, int scale_by_dA,
                            double* out, cudaStream_t s);
// per-instance maximum of the mode-2 partials
cudaError_t launch_finalize_max(const InstDev* insts, int n_inst, const double* partials, double* out,
                                cudaStream_t s);
// mode 0: C(a)/dA partials; mode 1: <a, b> partials; mode 2: max |a| partials
cudaError_t launch_field_reduce(int mode, const InstDev* insts, const int4* tiles, int ntiles, const double* a,
                                const double* b, double* partials, cudaStream_t s);
cudaError_t launch_field_axpby(const InstDev* insts, const int4* tiles, int ntiles, double* out,
                               const double* alpha, const double* a, const double* beta, const double* b,
                               cudaStream_t s);
// out = rho0(y) dA a (gradient of the constraint C at a), or with inverse
// != 0 out = a / (rho0(y) dA) (the representer of a in the energy inner product)
cudaError_t launch_field_weight(const InstDev* insts, const int4* tiles, int ntiles, double* out, const double* a,
                                int inverse, cudaStream_t s);
cudaError_t launch_localise(const InstDev* insts, const int4* tiles, int ntiles, double h_loc, double* v,
                            cudaStream_t s);

}  // namespace rt
