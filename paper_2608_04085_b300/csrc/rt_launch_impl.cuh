// rt_launch_impl.cuh -- launcher templates; included by one translation unit
// per state type, which instantiates them.
#pragma once

#include "rt_kernels.cuh"
#include "rt_launch.h"

namespace rt {

template <class T>
cudaError_t launch_inject(const InstDev* insts, const int4* tiles, int ntiles, const double* v, T* U,
                          const RunDev& run, int record, cudaStream_t s) {
  k_inject<T><<<ntiles, NTH, 0, s>>>(insts, tiles, v, U, run, record);
  return cudaGetLastError();
}

// tile variant with tiles of H rows; `tiles` is that height's work list
template <class T, int LIM, int H>
void launch_stage_tile(int stage, int mode, const InstDev* insts, const int4* tiles, int ntiles, const T* src,
                       const T* base, T* dst, const RunDev& run, int n, const TileMaps& tm, cudaStream_t s) {
  const size_t sm = StTile<H>::SMEM_ELEMS * sizeof(T);
  if (stage == 1) {
    k_stage_tile<T, 1, 2, LIM, H><<<ntiles, NTH, sm, s>>>(insts, tiles, src, base, dst, run, n, tm);
  } else if (mode == 0) {
    k_stage_tile<T, 2, 0, LIM, H><<<ntiles, NTH, sm, s>>>(insts, tiles, src, base, dst, run, n, tm);
  } else if (mode == 1) {
    k_stage_tile<T, 2, 1, LIM, H><<<ntiles, NTH, sm, s>>>(insts, tiles, src, base, dst, run, n, tm);
  } else {
    k_stage_tile<T, 2, 2, LIM, H><<<ntiles, NTH, sm, s>>>(insts, tiles, src, base, dst, run, n, tm);
  }
}

template <class T, int LIM>
cudaError_t launch_stage_lim(int variant, int stage, int mode, const InstDev* insts, const int4* strips, int nstrips,
                             const int4* tiles, int ntiles, const T* src, const T* base, T* dst, const RunDev& run,
                             int n, const TileMaps& tm, cudaStream_t s) {
  if (variant == STAGE_SWEEP) {
    const int grid = (nstrips + STRIP_WARPS - 1) / STRIP_WARPS, block = 32 * STRIP_WARPS;
    if (stage == 1) {  // stage 1 reads the recorded step constants in every mode
      k_stage_sweep<T, 1, 2, LIM><<<grid, block, 0, s>>>(insts, strips, nstrips, src, base, dst, run, n);
    } else if (mode == 0) {
      k_stage_sweep<T, 2, 0, LIM><<<grid, block, 0, s>>>(insts, strips, nstrips, src, base, dst, run, n);
    } else if (mode == 1) {
      k_stage_sweep<T, 2, 1, LIM><<<grid, block, 0, s>>>(insts, strips, nstrips, src, base, dst, run, n);
    } else {
      k_stage_sweep<T, 2, 2, LIM><<<grid, block, 0, s>>>(insts, strips, nstrips, src, base, dst, run, n);
    }
  } else if (variant == STAGE_TILE8) {
    launch_stage_tile<T, LIM, 8>(stage, mode, insts, tiles, ntiles, src, base, dst, run, n, tm, s);
  } else if (variant == STAGE_TILE32) {
    launch_stage_tile<T, LIM, 32>(stage, mode, insts, tiles, ntiles, src, base, dst, run, n, tm, s);
  } else {
    launch_stage_tile<T, LIM, 16>(stage, mode, insts, tiles, ntiles, src, base, dst, run, n, tm, s);
  }
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_stage(int variant, int lim, int stage, int mode, const InstDev* insts, const int4* strips,
                         int nstrips, const int4* tiles, int ntiles, const T* src, const T* base, T* dst,
                         const RunDev& run, int n, const TileMaps& tm, cudaStream_t s) {
  if (lim == LIM_MINMOD)
    return launch_stage_lim<T, LIM_MINMOD>(variant, stage, mode, insts, strips, nstrips, tiles, ntiles, src, base,
                                           dst, run, n, tm, s);
  return launch_stage_lim<T, -1>(variant, stage, mode, insts, strips, nstrips, tiles, ntiles, src, base, dst, run,
                                 n, tm, s);
}

template <class T, int AH>
void launch_adjoint_h(int lim, const InstDev* insts, const int4* tiles, int ntiles, const T* U, const T* K,
                      double kscale, const T* E, double escale, T* out, const RunDev& run, int n,
                      const TileMaps& tmu, const TileMaps& tmk, cudaStream_t s) {
  using G = AdjTile<AH>;
  const size_t sm = G::SMEM_ELEMS * sizeof(T);
  if (lim == LIM_MINMOD)
    k_adjoint<T, LIM_MINMOD, AH>
        <<<ntiles, G::NT, sm, s>>>(insts, tiles, U, K, (T)kscale, E, (T)escale, out, run, n, tmu, tmk);
  else
    k_adjoint<T, -1, AH><<<ntiles, G::NT, sm, s>>>(insts, tiles, U, K, (T)kscale, E, (T)escale, out, run, n, tmu,
                                                   tmk);
}

template <class T>
cudaError_t launch_adjoint(int rows, int lim, const InstDev* insts, const int4* tiles, int ntiles, const T* U,
                           const T* K, double kscale, const T* E, double escale, T* out, const RunDev& run, int n,
                           const TileMaps& tmu, const TileMaps& tmk, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (rows == 24) {
      launch_adjoint_h<T, 24>(lim, insts, tiles, ntiles, U, K, kscale, E, escale, out, run, n, tmu, tmk, s);
      return cudaGetLastError();
    }
  }
  if (rows != 16) return cudaErrorInvalidValue;
  launch_adjoint_h<T, 16>(lim, insts, tiles, ntiles, U, K, kscale, E, escale, out, run, n, tmu, tmk, s);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_objective(const InstDev* insts, const int4* tiles, int ntiles, T* const* slot_tab, int tab_mod,
                             const int* nstep, double* ek_out, T* lamA, T* lamB, double* partials,
                             cudaStream_t s) {
  k_objective<T><<<ntiles, NTH, 0, s>>>(insts, tiles, slot_tab, tab_mod, nstep, ek_out, lamA, lamB, partials);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_row_sums(const InstDev* insts, const int2* rows, int nrows, T* const* slot_tab, const int* nstep,
                            double2* out, cudaStream_t s) {
  k_row_sums<T><<<nrows, NTH, 0, s>>>(insts, rows, slot_tab, nstep, out);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_dt_partials(const InstDev* insts, const int4* tiles, int ntiles, const T* U, const T* U1,
                               const T* Un1, const T* lam, const T* lam1, const RunDev& run, int n, double* partials,
                               cudaStream_t s) {
  k_dt_partials<T><<<ntiles, NTH, 0, s>>>(insts, tiles, U, U1, Un1, lam, lam1, run, n, partials);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_dt_apply(const InstDev* insts, const int4* tiles, int ntiles, const T* U, T* lam, const RunDev& run,
                            int n, const double* coef, cudaStream_t s) {
  k_dt_apply<T><<<ntiles, NTH, 0, s>>>(insts, tiles, U, lam, run, n, coef);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_grad(const InstDev* insts, const int4* tiles, int ntiles, const T* lam, const double* v,
                        double* g, cudaStream_t s) {
  k_grad<T><<<ntiles, NTH, 0, s>>>(insts, tiles, lam, v, g);
  return cudaGetLastError();
}

template <class T, int LIM, int H>
cudaError_t configure_tile() {
  const int st = (int)(StTile<H>::SMEM_ELEMS * sizeof(T));
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(k_stage_tile<T, 1, 2, LIM, H>, a, st);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_stage_tile<T, 2, 0, LIM, H>, a, st);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_stage_tile<T, 2, 1, LIM, H>, a, st);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_stage_tile<T, 2, 2, LIM, H>, a, st);
  return e;
}

template <class T, int LIM>
cudaError_t configure_lim() {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = configure_tile<T, LIM, 8>();
  if (e == cudaSuccess) e = configure_tile<T, LIM, 16>();
  if (e == cudaSuccess) e = configure_tile<T, LIM, 32>();
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_adjoint<T, LIM, 16>, a, (int)(AdjTile<16>::SMEM_ELEMS * sizeof(T)));
  if constexpr (sizeof(T) == 4)
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_adjoint<T, LIM, 24>, a, (int)(AdjTile<24>::SMEM_ELEMS * sizeof(T)));
  return e;
}

template <class T>
cudaError_t configure_kernels() {
  cudaError_t e = configure_lim<T, LIM_MINMOD>();
  if (e == cudaSuccess) e = configure_lim<T, -1>();
  return e;
}

#define RT_INSTANTIATE_LAUNCHERS(T)                                                                              \
  template cudaError_t launch_inject<T>(const InstDev*, const int4*, int, const double*, T*, const RunDev&, int,  \
                                        cudaStream_t);                                                           \
  template cudaError_t launch_stage<T>(int, int, int, int, const InstDev*, const int4*, int, const int4*, int,    \
                                       const T*, const T*, T*, const RunDev&, int, const TileMaps&,              \
                                       cudaStream_t);                                                            \
  template cudaError_t launch_adjoint<T>(int, int, const InstDev*, const int4*, int, const T*, const T*, double,  \
                                         const T*, double, T*, const RunDev&, int, const TileMaps&,              \
                                         const TileMaps&, cudaStream_t);                                         \
  template cudaError_t launch_objective<T>(const InstDev*, const int4*, int, T* const*, int, const int*, double*, \
                                           T*, T*, double*, cudaStream_t);                                       \
  template cudaError_t launch_grad<T>(const InstDev*, const int4*, int, const T*, const double*, double*,         \
                                      cudaStream_t);                                                             \
  template cudaError_t launch_row_sums<T>(const InstDev*, const int2*, int, T* const*, const int*, double2*,       \
                                          cudaStream_t);                                                         \
  template cudaError_t launch_dt_partials<T>(const InstDev*, const int4*, int, const T*, const T*, const T*,      \
                                             const T*, const T*, const RunDev&, int, double*, cudaStream_t);      \
  template cudaError_t launch_dt_apply<T>(const InstDev*, const int4*, int, const T*, T*, const RunDev&, int,     \
                                          const double*, cudaStream_t);                                          \
  template cudaError_t configure_kernels<T>();

}  // namespace rt
