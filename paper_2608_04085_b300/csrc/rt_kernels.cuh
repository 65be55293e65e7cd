// rt_kernels.cuh -- CUDA kernels of the hot path, templated on the state type.
//
// One CTA advances one tile of TILE_X x TILE_Y cells of one instance (two
// cells per thread); the tile list covers every instance of the batch, so a
// single launch advances all instances, uniform or uneven grids alike. The
// per-instance time-step control lives on the device: the last CTA of an
// instance in each stage-2 launch turns the CFL minimum into the next dt and
// the next step's constants, so the kernels do no FP64 arithmetic per cell
// and the host never reads dt inside the time loop.
//
// An FP64 state slot holds U; an FP32 slot holds U - U_b(y), the deviation
// from the hydrostatic base U_b = (rho0, 0, 0, p0/(gamma-1)) of the cell's
// row (state_to_prim adds the base back), so FP32 rounding is relative to the
// perturbation rather than to the O(1) background. Both run the same scheme.
//
//   k_inject     Sec. 3.1: U0 = (rho0, rho0 v, p0/(gamma-1) + rho0|v|^2/2), first CFL minimum
//   k_stage_*<1> U1 = U + dt L(U)                       (SSP-RK2 stage 1)
//   k_stage_*<2> U' = U/2 + (U1 + dt L(U1))/2           (stage 2) + CFL minimum of U'
//                L(U): finite-volume divergence of PLM+HLLC fluxes + gravity
//                source (Sec. 2.1 Eqs. mass/momentum/energy, Sec. 2.3);
//                a warp-sweep variant and a shared-memory tile variant.
//   k_adjoint    out = kap + (d(dt L)/dU)^T kap + escale*E, kap = kscale*K: the
//                transposed stage map (Sec. 3.4, exact discrete gradient)
//   k_objective  J = sum e_k dA and sum (e_k - e_k0)^2 dA (Eqs. ke, objective),
//                optional terminal cotangent dJ/dU
//   k_grad       dJ/dv from dJ/dU0 (transpose of k_inject)
//   k_field_*    constraint C (Eq. constraint), dot products, axpby (projection)
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rt_internal.h"
#include "rt_scheme.cuh"

namespace rt {

constexpr int TX = TILE_X, TY = TILE_Y, NTH = TILE_THREADS;
constexpr int ROWS_PER_PASS = NTH / TX;  // rows covered by one pass of the block over a tile
static_assert(TX == 32, "one warp per tile row");
static_assert(TY % ROWS_PER_PASS == 0, "tile rows must be a multiple of the rows per pass");

// Periodic x index; one correction covers every tile offset when nx is at
// least the halo width, the modulo handles the rest.
__device__ __forceinline__ int wrap_x(int gx, int nx) {
  if (gx < 0) gx += nx;
  else if (gx >= nx) gx -= nx;
  if (gx < 0 || gx >= nx) {
    gx %= nx;
    if (gx < 0) gx += nx;
  }
  return gx;
}

// Offset of row gy (a held row of the instance) inside one perturbation
// component: rows count from the instance's first owned row.
__device__ __forceinline__ long long vrow(const InstDev& I, int gy) { return (long long)(gy - I.own0) * I.nx; }

// The 4th component of a tile or strip descriptor packs the problem index
// (bits 0-23) and the descriptor's rows to compute (bits 24-31, at most the
// tile height): the hot kernels bound their rows and select the problem's run
// scalars from data they already hold.
__device__ __forceinline__ int desc_run(int w) { return w & 0xffffff; }
__device__ __forceinline__ int desc_rows(int w) { return (int)((unsigned)w >> 24); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum in a fixed order (deterministic); the result is valid in
// thread 0. All threads must call.
__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

// Block-wide maximum of non-negative values (result in thread 0).
__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = fmax(s, red[w]);
  return s;
}

// Physics constants of an instance in the state precision (no conversion
// instructions in the kernels).
template <class T>
struct Phys {
  T gamma, gm1, g, dx, dy;
};
template <class T> __device__ __forceinline__ Phys<T> phys(const InstDev& I);
template <> __device__ __forceinline__ Phys<float> phys<float>(const InstDev& I) {
  return {I.gamma_f, I.gm1_f, I.g_f, I.dx_f, I.dy_f};
}
template <> __device__ __forceinline__ Phys<double> phys<double>(const InstDev& I) {
  return {I.gamma, I.gm1, I.g_y, I.dx, I.dy};
}

// Riemann-flux choice of instance I in a kernel built for limiter LIM: the
// limiter-specialised kernels (LIM >= 0) run HLLC only (the runtime sends
// batches with another flux to the generic LIM = -1 kernels).
template <class T, int LIM>
__device__ __forceinline__ FluxSel<T> flux_sel(const InstDev& I) {
  if constexpr (LIM >= 0) {
    return {FLUX_HLLC, T(0)};
  } else if constexpr (sizeof(T) == 4) {
    return {I.flux, I.flux_theta_f};
  } else {
    return {I.flux, I.flux_theta};
  }
}

template <class T>
__device__ __forceinline__ StepC<T> step_const(const RunDev& run, int inst, int n) {
  return reinterpret_cast<const StepC<T>*>(run.dtc)[(long long)inst * run.max_steps + n];
}

// The row's base (rho0, p0) as the FP32 conversion uses it (unused for FP64).
struct RowBase {
  float rho, p;
};

template <class T>
__device__ __forceinline__ RowBase row_base(const InstDev& I, int row) {
  if constexpr (sizeof(T) == 4) return {__ldg(I.rho0_f + row), __ldg(I.p0_f + row)};
  else return {0.f, 0.f};
}

// Stored state -> primitives (rho, u_x, u_y, p) of a cell whose row has the
// base b. An FP64 state stores U itself. An FP32 state stores the deviation
// of U from the row's hydrostatic base (rho0, 0, 0, p0/(gamma-1)): the stored
// values and every update then round relative to the deviation, not to the
// O(1) background, and the primitives add the base back: rho = rho0 + d_rho,
// p = p0 + (gamma-1)(d_E - |m|^2/(2 rho)). In exact arithmetic both give the
// same scheme.
template <class T>
__device__ __forceinline__ void state_to_prim_b(T s0, T s1, T s2, T s3, RowBase b, T gm1, T W[4]) {
  if constexpr (sizeof(T) == 4) {
    const T r = s0 + b.rho;
    W[0] = r;
    W[1] = s1 / r;
    W[2] = s2 / r;
    W[3] = b.p + gm1 * (s3 - T(0.5) * (s1 * W[1] + s2 * W[2]));
  } else {
    cons_to_prim(s0, s1, s2, s3, gm1, W);
  }
}

template <class T>
__device__ __forceinline__ void state_to_prim(T s0, T s1, T s2, T s3, const InstDev& I, int row, T gm1, T W[4]) {
  state_to_prim_b(s0, s1, s2, s3, row_base<T>(I, row), gm1, W);
}

// Full density from the stored density and the row's base.
template <class T>
__device__ __forceinline__ T state_rho(T s0, RowBase b) {
  if constexpr (sizeof(T) == 4) return s0 + b.rho;
  else return s0;
}

// Full density and pressure in FP64 from a stored state (diagnostics and the
// step-control derivative).
template <class T>
__device__ __forceinline__ void state_rho_p_f64(T s0, T s1, T s2, T s3, const InstDev& I, int row, double& rho,
                                                double& p) {
  const double m1 = s1, m2 = s2;
  if constexpr (sizeof(T) == 4) {
    rho = (double)s0 + (double)I.rho0_f[row];
    p = (double)I.p0_f[row] + I.gm1 * ((double)s3 - 0.5 * (m1 * (m1 / rho) + m2 * (m2 / rho)));
  } else {
    rho = s0;
    p = I.gm1 * (s3 - 0.5 * (m1 * (m1 / rho) + m2 * (m2 / rho)));
  }
}

// Cell crossing time min(dx/(|u_x|+c), dy/(|u_y|+c)) of a conserved state in
// the state's precision; `bad` flags a non-positive density or pressure, or
// a NaN.
template <class T>
__device__ __forceinline__ T crossing_time(T s0, T s1, T s2, T s3, RowBase rb, const Phys<T>& P, bool& bad) {
  T W[4];
  state_to_prim_b(s0, s1, s2, s3, rb, P.gm1, W);
  const T c = sqrt(P.gamma * W[3] / W[0]);
  const T wx = P.dx / (fabs(W[1]) + c);
  const T wy = P.dy / (fabs(W[2]) + c);
  const T w = wx <= wy ? wx : wy;
  bad = !(W[0] > T(0)) || !(W[3] > T(0)) || !(w > T(0)) || !(w < T(1e30));
  return w;
}

template <class T>
__device__ __forceinline__ T warp_min_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u < v ? u : v;
  }
  return v;
}

// Time-step control of step n_next (thread 0 of the instance's last CTA):
// dt = cfl * min crossing time, clipped to T - t in horizon mode, 0 once the
// run is over or the state went bad. Resets the running minimum.
template <class T>
__device__ void finish_step(const InstDev& I, const RunDev& run, int inst, int n_next, double t) {
  const unsigned long long bits = atomicExch(&run.wmin[inst], ~0ull);
  const double wmin = __longlong_as_double((long long)bits);
  const bool ok = atomicAdd(&run.status[inst], 0) == 0 && bits != ~0ull;
  const bool active = ok && I.enabled && (I.nsteps > 0 ? n_next < I.nsteps : t < I.T);
  double dt = I.cfl * wmin;
  bool clipped = false;
  if (I.nsteps <= 0) {
    const double rem = I.T - t;
    if (dt >= rem) {
      dt = rem;
      clipped = true;
    }
  }
  if (!active) dt = 0.0;
  if (n_next < run.max_steps) {
    const long long k = (long long)inst * run.max_steps + n_next;
    run.dtrec[k] = dt;
    run.wrec[k] = !active ? 0.0 : (clipped ? -1.0 : wmin);
    StepC<T> c;
    c.dt = (T)dt;
    c.dtdx = (T)(dt / I.dx);
    c.dtdy = (T)(dt / I.dy);
    c.dtg = (T)(dt * I.g_y);
    reinterpret_cast<StepC<T>*>(run.dtc)[k] = c;
  }
}

// Fold the block's crossing-time minimum into the instance's running minimum
// and report whether this CTA is the instance's last one of the launch.
// All threads must call; the result is valid in thread 0.
template <class T>
__device__ __forceinline__ bool commit_crossing(T w, long long cell, bool bad, int ntile_run, const RunDev& run,
                                                int inst, T* red) {
  if (bad) {
    if (atomicCAS(&run.status[inst], 0, 1) == 0) run.bad_cell[inst] = cell;
  }
  T m = warp_min_t(w);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = m;
  __syncthreads();
  bool last = false;
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) m = red[k] < m ? red[k] : m;
    if (m > T(0) && m < T(1e30))
      atomicMin(&run.wmin[inst], (unsigned long long)__double_as_longlong((double)m));
    __threadfence();
    if (atomicAdd(&run.counter[inst], 1u) + 1u == (unsigned int)ntile_run) {
      run.counter[inst] = 0u;
      __threadfence();
      last = true;
    }
  }
  return last;
}

// ------------------------------------------------------------------ inject
template <class T>
__global__ void __launch_bounds__(NTH) k_inject(const InstDev* __restrict__ insts, const int4* __restrict__ tiles,
                                                const double* __restrict__ v, T* __restrict__ U, RunDev run,
                                                int record) {
  __shared__ T red[NTH / 32];
  const int4 tl = tiles[blockIdx.x];
  const InstDev& I = insts[tl.x];
  const int inst = desc_run(tl.w);
  const Phys<T> P = phys<T>(I);
  const long long cells = (long long)I.nx * I.ny;
  T w = T(1e30);
  bool bad = false;
  long long badc = 0;
  for (int e = threadIdx.x; e < TX * TY; e += NTH) {
    const int gx = tl.y + e % TX, gy = tl.z + e / TX;
    if (gx >= I.nx || gy >= I.own1) continue;
    const long long c = (long long)gy * I.nx + gx;
    const double* vi = v + I.v_off + vrow(I, gy) + gx;
    const double vx = I.ncomp == 2 ? vi[0] : 0.0;
    const double vy = I.ncomp == 2 ? vi[I.v_plane] : vi[0];
    const double r0 = I.rho0[gy], p0 = I.p0[gy];
    T* Ui = U + 4 * I.cell_off;
    // an FP32 state stores the deviation from the row's base (state_to_prim)
    const double rb = sizeof(T) == 4 ? (double)I.rho0_f[gy] : 0.0;
    const double pb = sizeof(T) == 4 ? (double)I.p0_f[gy] : 0.0;
    const T u0 = (T)(r0 - rb), u1 = (T)(r0 * vx), u2 = (T)(r0 * vy);
    const T u3 = (T)((p0 - pb) / I.gm1 + 0.5 * r0 * (vx * vx + vy * vy));
    Ui[c] = u0;
    Ui[cells + c] = u1;
    Ui[2 * cells + c] = u2;
    Ui[3 * cells + c] = u3;
    bool b = false;
    const T cw = crossing_time<T>(u0, u1, u2, u3, row_base<T>(I, gy), P, b);
    if (b) { bad = true; badc = c; } else if (cw < w) w = cw;
  }
  if (commit_crossing<T>(w, badc, bad, I.run_tiles, run, inst, red)) {
    run.t[inst] = 0.0;
    run.nstep[inst] = 0;
    if (record) finish_step<T>(I, run, inst, 0, 0.0);  // a replay keeps the recorded step 0
  }
}

// ------------------------------------------------------------------- stage
// Two variants of one stage kernel compute the same values bit for bit; the
// runtime's autotuner picks the faster for the batch at hand. LIM >= 0 fixes
// the limiter at compile time (every instance of the batch uses it); -1
// reads each instance's limiter.
//
// Sweep variant: each warp advances one strip of STRIP_W x STRIP_H cells,
// marching up the rows. Lane L holds column x0 - 2 + L; the y direction keeps
// a two-row window of primitive states, the y slope of the current row and
// the flux through the current row's bottom face in registers; the x
// neighbours come from warp shuffles. Every slope and every face flux is
// evaluated once; no shared memory, no block barrier.
//
// MODE 0: CFL control (the instance's last warp records the next dt, advances
// t and the step count); MODE 1: replay recorded steps, counting them;
// MODE 2: replay without touching any run scalar (checkpoint recomputation).
template <class T>
__device__ __forceinline__ T shfl_up1(T v) { return __shfl_up_sync(0xffffffffu, v, 1); }
template <class T>
__device__ __forceinline__ T shfl_down1(T v) { return __shfl_down_sync(0xffffffffu, v, 1); }

// Conserved values of row r of column gcol as the sweep needs them: the
// row itself, or for a ghost row the interior row it mirrors (the primitive
// transform is applied by raw_to_prim). Rows beyond the ghost layers get a
// harmless placeholder.
template <class T>
__device__ __forceinline__ void load_raw(const T* __restrict__ Ui, int nx, int ny, long long cells, int gcol, int r,
                                         T u[4]) {
  int sy = r;
  if (r < 0) sy = -1 - r;
  else if (r >= ny) sy = 2 * ny - 1 - r;
  if (sy < 0 || sy >= ny) {
    u[0] = T(1); u[1] = T(0); u[2] = T(0); u[3] = T(1);
    return;
  }
  const long long c = (long long)sy * nx + gcol;
  u[0] = Ui[c];
  u[1] = Ui[cells + c];
  u[2] = Ui[2 * cells + c];
  u[3] = Ui[3 * cells + c];
}

// Interior row whose base state row r uses: r itself, the row a ghost row
// mirrors, or (rows beyond the ghost layers, which hold load_raw's
// placeholder) the nearest interior row.
__device__ __forceinline__ int base_row(int r, int ny) {
  int sy = r;
  if (r < 0) sy = -1 - r;
  else if (r >= ny) sy = 2 * ny - 1 - r;
  return sy < 0 ? 0 : (sy >= ny ? ny - 1 : sy);
}

// Primitive state of row r from load_raw's values and the base of
// base_row(r), with the y boundary conditions applied: ghost rows mirror the
// interior (u_y negated) and, for the hydrostatic boundary, extrapolate
// p_g = p_c + g_y rho_c (y_g - y_c).
template <class T>
__device__ __forceinline__ void raw_to_prim(const T u[4], const InstDev& I, int r, RowBase rb, const Phys<T>& P,
                                            T W[4]) {
  int side = 0, k = 0;
  if (r < 0) { side = -1; k = -1 - r; }
  else if (r >= I.ny) { side = 1; k = r - I.ny; }
  state_to_prim_b(u[0], u[1], u[2], u[3], rb, P.gm1, W);
  if (side != 0) {
    W[2] = -W[2];
    if (I.bc_y == 1) {
      const T dyk = (T)((double)(2 * k + 1) * I.dy);
      if (side < 0) W[3] = W[3] - P.g * W[0] * dyk;
      else W[3] = W[3] + P.g * W[0] * dyk;
    }
  }
}

// Load a tile of primitive states into shared memory (layout [4][EY][EX],
// origin (gx0, gy0)), issuing every global load of this thread's cells before
// converting any of them, so that they are in flight together.
// Four values of one cell held together (one 16-byte shared-memory access
// for FP32, two for FP64).
template <class T>
struct __align__(16) Q4 {
  T v[4];
};

// INTERIOR: the tile with its ghost layers lies inside the grid (no periodic
// wrap, no mirrored wall rows), so cells are addressed directly.
template <class T, int EX, int EY, bool AOS, bool INTERIOR, int NT = NTH>
__device__ __forceinline__ void load_prim_tile_impl(const T* __restrict__ Ui, const InstDev& I, long long cells,
                                                    int gx0, int gy0, const Phys<T>& P, T* __restrict__ sW,
                                                    RowBase* __restrict__ sRB) {
  constexpr int N = EX * EY;
  constexpr int PER = (N + NT - 1) / NT;
  static_assert(EY <= NT, "one thread per tile row fills the base table");
  // FP32: the base of every tile row, loaded together with the state, stored
  // once the state loads are issued and read back after the barrier
  RowBase rbv{0.f, 0.f};
  if (sizeof(T) == 4 && threadIdx.x < EY) rbv = row_base<T>(I, base_row(gy0 + threadIdx.x, I.ny));
  T u[PER][4];
  int rr[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int e = threadIdx.x + k * NT;
    rr[k] = 0;
    if (e < N) {
      const int ey = e / EX, ex = e - ey * EX;
      rr[k] = gy0 + ey;
      if (INTERIOR) {
        const T* p = Ui + ((long long)rr[k] * I.nx + gx0 + ex);
#pragma unroll
        for (int q = 0; q < 4; ++q) u[k][q] = p[q * cells];
      } else {
        load_raw(Ui, I.nx, I.ny, cells, wrap_x(gx0 + ex, I.nx), rr[k], u[k]);
      }
    }
  }
  if (sizeof(T) == 4) {
    if (threadIdx.x < EY) sRB[threadIdx.x] = rbv;
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int e = threadIdx.x + k * NT;
    if (e < N) {
      const int ey = e / EX, ex = e - ey * EX;
      T W[4];
      const RowBase rb = sizeof(T) == 4 ? sRB[ey] : RowBase{0.f, 0.f};
      if (INTERIOR) state_to_prim_b(u[k][0], u[k][1], u[k][2], u[k][3], rb, P.gm1, W);
      else raw_to_prim(u[k], I, rr[k], rb, P, W);
      if (AOS) {
        Q4<T> c;
#pragma unroll
        for (int q = 0; q < 4; ++q) c.v[q] = W[q];
        reinterpret_cast<Q4<T>*>(sW)[ey * EX + ex] = c;
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) sW[(q * EY + ey) * EX + ex] = W[q];
      }
    }
  }
}

// Load a tile of primitive states (see load_prim_tile_impl); the interior
// case, decided once for the whole CTA, skips the boundary logic.
template <class T, int EX, int EY, bool AOS = false, int NT = NTH>
__device__ __forceinline__ void load_prim_tile(const T* __restrict__ Ui, const InstDev& I, long long cells, int gx0,
                                               int gy0, const Phys<T>& P, T* __restrict__ sW,
                                               RowBase* __restrict__ sRB) {
  if (gx0 >= 0 && gx0 + EX <= I.nx && gy0 >= 0 && gy0 + EY <= I.ny)
    load_prim_tile_impl<T, EX, EY, AOS, true, NT>(Ui, I, cells, gx0, gy0, P, sW, sRB);
  else
    load_prim_tile_impl<T, EX, EY, AOS, false, NT>(Ui, I, cells, gx0, gy0, P, sW, sRB);
}

// ------------------------------------------------------------- TMA tile loads
// One thread initialises an mbarrier, announces the bytes to expect and
// issues one cp.async.bulk.tensor copy per box; every thread then waits on
// the barrier's phase 0 (once per CTA) before reading the staged boxes.

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// First 128-byte boundary at or after p (the staging areas have the slack).
template <class T>
__device__ __forceinline__ T* align128(void* p) {
  const uint32_t a = smem_addr(p);
  return reinterpret_cast<T*>(static_cast<unsigned char*>(p) + ((128u - (a & 127u)) & 127u));
}

__device__ __forceinline__ void mbar_init_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// Box (x, y, component 0, instance z) of the map's tensor into dst.
__device__ __forceinline__ void tma_box(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
      "%5}], [%6];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(0), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// Poll phase `parity` of the barrier at most `limit` times, each poll
// suspending the thread for at most TMA_POLL_NS nanoseconds while the phase
// is incomplete; false if it never completed.
constexpr int TMA_POLL_NS = 1000;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit) {
  for (int i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, "
        "p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity), "n"(TMA_POLL_NS)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Wait for this CTA's TMA boxes, at most run.tma_polls polls (2^18, about a
// quarter of a second). A wait that gives up records status 2 for the
// problem (the host reports RT_ETIMEOUT) and waits once more, again bounded,
// for copies still in flight; the CTA then finishes on whatever the staging
// area holds, so the launch always ends.
__device__ __forceinline__ void tma_wait(uint64_t* bar, const RunDev& run, int inst) {
  if (!mbar_wait(bar, 0, run.tma_polls)) {
    atomicCAS(&run.status[inst], 0, 2);
    mbar_wait(bar, 0, run.tma_polls);
  }
}

// A tile takes its box from TMA: the instance belongs to a TMA group and the
// box (TMA_BOX_X columns from x0 - 4, rows y0 - gy .. y0 + rows + gy - 1)
// lies inside the held rows and columns. Tiles at the periodic seam or a
// wall keep the plain loads, whose per-cell wrap and mirror logic TMA cannot
// express (a box with that logic done afterwards measured slower).
__device__ __forceinline__ bool tma_tile(const InstDev& I, int x0, int y0, int rows, int gy) {
  return I.tma_g >= 0 && x0 >= 4 && x0 - 4 + TMA_BOX_X <= I.nx && y0 >= gy && y0 + rows + gy <= I.ny;
}

// Staged box [4][BY][TMA_BOX_X] -> tile of primitive states (cell-major Q4)
// of EX x EY cells starting at column `ox` of the box and at its first row;
// the box lies inside the grid (tma_tile). sRB holds the base of every box
// row (FP32).
template <class T, int EX, int EY, int BY, int NT = NTH>
__device__ __forceinline__ void prim_from_box(const T* __restrict__ box, int ox, const Phys<T>& P,
                                              const RowBase* __restrict__ sRB, Q4<T>* __restrict__ sW) {
  constexpr int N = EX * EY, PER = (N + NT - 1) / NT, PL = BY * TMA_BOX_X;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int e = threadIdx.x + k * NT;
    if (e < N) {
      const int ey = e / EX, ex = e - ey * EX;
      const T* b = box + ey * TMA_BOX_X + ex + ox;
      const RowBase rb = sizeof(T) == 4 ? sRB[ey] : RowBase{0.f, 0.f};
      T W[4];
      state_to_prim_b(b[0], b[PL], b[2 * PL], b[3 * PL], rb, P.gm1, W);
      Q4<T> c;
#pragma unroll
      for (int q = 0; q < 4; ++q) c.v[q] = W[q];
      sW[e] = c;
    }
  }
}

template <class T, int STAGE, int MODE, int LIM>
__global__ void __launch_bounds__(32 * STRIP_WARPS, 6) k_stage_sweep(const InstDev* __restrict__ insts,
                                                            const int4* __restrict__ strips, int nstrips,
                                                            const T* __restrict__ src, const T* __restrict__ base,
                                                            T* __restrict__ dst, RunDev run, int n) {
  const int lane = threadIdx.x & 31;
  const int si = blockIdx.x * STRIP_WARPS + (threadIdx.x >> 5);
  if (si >= nstrips) return;  // the whole warp leaves; no block-level synchronisation below
  const int4 st = strips[si];
  const InstDev& I = insts[st.x];
  const int inst = desc_run(st.w);
  const StepC<T> sc = step_const<T>(run, inst, n);
  if (!(sc.dt > T(0))) return;  // instance inactive at this step (uniform over the warp)

  const Phys<T> P = phys<T>(I);
  const int nx = I.nx, ny = I.ny, lim = LIM >= 0 ? LIM : I.limiter;
  const FluxSel<T> fs = flux_sel<T, LIM>(I);
  const long long cells = (long long)nx * ny;
  const T* Si = src + 4 * I.cell_off;
  const T* Bi = base + 4 * I.cell_off;
  T* Di = dst + 4 * I.cell_off;
  const int x0 = st.y, y0 = st.z;
  const int col = x0 - 2 + lane;
  const int gcol = wrap_x(col, nx);
  const bool writer = lane >= 2 && lane < 2 + STRIP_W && col < nx;
  const int y1 = y0 + desc_rows(st.w);

  // prologue: rows y0-2 .. y0+2, y slopes of rows y0-1 and y0, flux through
  // the bottom face of row y0
  T Ua[4], Ub[4], U0[4], U1[4], U2[4];
  load_raw(Si, nx, ny, cells, gcol, y0 - 2, Ua);
  load_raw(Si, nx, ny, cells, gcol, y0 - 1, Ub);
  load_raw(Si, nx, ny, cells, gcol, y0, U0);
  load_raw(Si, nx, ny, cells, gcol, y0 + 1, U1);
  load_raw(Si, nx, ny, cells, gcol, y0 + 2, U2);
  T W0[4], W1[4], s_cur[4], Gb[4];
  {
    T Wa[4], Wb[4], WL[4], WR[4];
    raw_to_prim(Ua, I, y0 - 2, row_base<T>(I, base_row(y0 - 2, ny)), P, Wa);
    raw_to_prim(Ub, I, y0 - 1, row_base<T>(I, base_row(y0 - 1, ny)), P, Wb);
    raw_to_prim(U0, I, y0, row_base<T>(I, base_row(y0, ny)), P, W0);
    raw_to_prim(U1, I, y0 + 1, row_base<T>(I, base_row(y0 + 1, ny)), P, W1);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T s_lo = limited_slope(Wa[q], Wb[q], W0[q], lim);
      s_cur[q] = limited_slope(Wb[q], W0[q], W1[q], lim);
      WL[q] = Wb[q] + T(0.5) * s_lo;
      WR[q] = W0[q] - T(0.5) * s_cur[q];
    }
    face_flux_states<T, 1>(WL, WR, P.gamma, P.gm1, fs, Gb);
  }

  T wmin = T(1e30);
  bool bad = false;
  long long badc = 0;
  for (int j = y0; j < y1; ++j) {
    // prefetch row j+3 and, for stage 2, the base state of row j
    T U3[4], B0[4];
    load_raw(Si, nx, ny, cells, gcol, j + 3, U3);
    const long long c = (long long)j * nx + col;
    if (STAGE == 2) {
      if (writer) {
#pragma unroll
        for (int k = 0; k < 4; ++k) B0[k] = Bi[k * cells + c];
      } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) B0[k] = T(0);
      }
    }
    const RowBase rbj = row_base<T>(I, j);
    // x face on the left of this lane's cell in row j
    T Fl[4];
    {
      T WL[4], WR[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const T wm = shfl_up1(W0[q]), wp = shfl_down1(W0[q]);
        const T sx = limited_slope(wm, W0[q], wp, lim);
        WL[q] = shfl_up1(W0[q] + T(0.5) * sx);
        WR[q] = W0[q] - T(0.5) * sx;
      }
      face_flux_states<T, 0>(WL, WR, P.gamma, P.gm1, fs, Fl);
    }
    T Fr[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) Fr[q] = shfl_down1(Fl[q]);
    // y face between rows j and j+1
    T W2[4], s_next[4], Gt[4];
    raw_to_prim(U2, I, j + 2, row_base<T>(I, base_row(j + 2, ny)), P, W2);
    {
      T WL[4], WR[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        s_next[q] = limited_slope(W0[q], W1[q], W2[q], lim);
        WL[q] = W0[q] + T(0.5) * s_cur[q];
        WR[q] = W1[q] - T(0.5) * s_next[q];
      }
      face_flux_states<T, 1>(WL, WR, P.gamma, P.gm1, fs, Gt);
    }
    if (writer) {
      T o[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        T b = U0[k] + sc.dtdx * (Fl[k] - Fr[k]);
        b = b + sc.dtdy * (Gb[k] - Gt[k]);
        if (k == 2) b = b + sc.dt * (state_rho(U0[0], rbj) * P.g);
        if (k == 3) b = b + sc.dt * (U0[2] * P.g);
        o[k] = STAGE == 2 ? T(0.5) * B0[k] + T(0.5) * b : b;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) Di[k * cells + c] = o[k];
      if (STAGE == 2 && MODE == 0) {
        bool b = false;
        const T cw = crossing_time<T>(o[0], o[1], o[2], o[3], rbj, P, b);
        if (b) { bad = true; badc = c; } else if (cw < wmin) wmin = cw;
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      W0[q] = W1[q];
      W1[q] = W2[q];
      U0[q] = U1[q];
      U1[q] = U2[q];
      U2[q] = U3[q];
      s_cur[q] = s_next[q];
      Gb[q] = Gt[q];
    }
  }

  if (STAGE == 2 && MODE == 0) {
    if (bad) {
      if (atomicCAS(&run.status[inst], 0, 1) == 0) run.bad_cell[inst] = badc;
    }
    const T m = warp_min_t(wmin);
    if (lane == 0) {
      if (m > T(0) && m < T(1e30))
        atomicMin(&run.wmin[inst], (unsigned long long)__double_as_longlong((double)m));
      __threadfence();
      const unsigned int nst = (unsigned int)I.run_strips;
      if (atomicAdd(&run.counter[inst], 1u) + 1u == nst) {
        run.counter[inst] = 0u;
        __threadfence();
        const double dt = run.dtrec[(long long)inst * run.max_steps + n];
        const double t = run.t[inst];
        const double tn = I.nsteps > 0 ? t + dt : (dt >= I.T - t ? I.T : t + dt);
        run.t[inst] = tn;
        run.nstep[inst] = n + 1;
        finish_step<T>(I, run, inst, n + 1, tn);
      }
    }
  }
  if (STAGE == 2 && MODE == 1 && x0 == 0 && y0 == 0 && lane == 0) run.nstep[inst] = n + 1;
}

// --------------------------------------------------------- stage (tile variant)
// Shared memory, cell-major (the 4 values of a cell or face together, Q4):
// primitive tile with 2 ghost layers, x-face and y-face fluxes.
// Geometry of a tile of H rows (32 columns).
template <int H>
struct StTile {
  static constexpr int EX = TX + 4, EY = H + 4;
  static constexpr int NFX = (TX + 1) * H, NFY = TX * (H + 1);
  static constexpr int SMEM_ELEMS = 4 * EX * EY + 4 * NFX + 4 * NFY;
  static constexpr int PASSES = (H + ROWS_PER_PASS - 1) / ROWS_PER_PASS;
  static constexpr int LIST = H == 8 ? 0 : (H == 16 ? 1 : 2);  // index into InstDev::run_tiles_h
};

// Tile variant of the stage kernel: one CTA of 256 threads per tile of 32
// columns and H = 8, 16 or 32 rows, primitive states with 2 ghost layers in
// shared memory, one thread per face, then one thread per cell for the
// update. Modes as for the sweep variant. FP32 launches are held to 6 CTAs per
// SM for H <= 16 (40 registers) and 4 for H = 32, which the stage-2 variant
// with the step control would otherwise exceed.
template <class T, int STAGE, int MODE, int LIM, int H>
__global__ void __launch_bounds__(NTH, sizeof(T) == 4 ? (H <= 16 ? 6 : 4) : 1) k_stage_tile(const InstDev* __restrict__ insts, const int4* __restrict__ tiles,
                                               const T* __restrict__ src, const T* __restrict__ base,
                                               T* __restrict__ dst, RunDev run, int n,
                                               const __grid_constant__ TileMaps tm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using G = StTile<H>;
  Q4<T>* sW = reinterpret_cast<Q4<T>*>(smem_raw);  // [EY][EX]
  Q4<T>* sF = sW + G::EX * G::EY;                  // [H][TX+1]
  Q4<T>* sG = sF + G::NFX;                         // [H+1][TX]
  __shared__ T red[NTH / 32];
  __shared__ RowBase sRB[G::EY];
  __shared__ __align__(8) uint64_t s_bar;
  const int4 tl = tiles[blockIdx.x];
  const InstDev& I = insts[tl.x];
  const int inst = desc_run(tl.w);
  const StepC<T> sc = step_const<T>(run, inst, n);
  if (!(sc.dt > T(0))) return;  // instance inactive at this step (uniform over the block)

  const Phys<T> P = phys<T>(I);
  const long long cells = (long long)I.nx * I.ny;
  const T* Si = src + 4 * I.cell_off;
  const int x0 = tl.y, y0 = tl.z;
  const int lim = LIM >= 0 ? LIM : I.limiter;
  const FluxSel<T> fs = flux_sel<T, LIM>(I);
  // the primitive tile: from a TMA box staged in the (not yet used) face
  // buffers, or by plain loads
  constexpr int BOX = 4 * G::EY * TMA_BOX_X;
  static_assert((G::NFX + G::NFY) * 4 >= BOX + 128 / sizeof(T), "staging area too small");
  const bool tma = tma_tile(I, x0, y0, H, 2);
  T* box = align128<T>(sF);
  if (tma) {
    if (threadIdx.x == 0) {
      mbar_init_expect(&s_bar, BOX * sizeof(T));
      if (!run.tma_skip) tma_box(box, &tm.m[I.tma_g], x0 - 4, y0 - 2, I.tma_z, &s_bar);
    }
    if (sizeof(T) == 4 && threadIdx.x < G::EY) sRB[threadIdx.x] = row_base<T>(I, y0 - 2 + threadIdx.x);
  } else {
    load_prim_tile<T, G::EX, G::EY, true>(Si, I, cells, x0 - 2, y0 - 2, P, reinterpret_cast<T*>(sW), sRB);
  }
  // stage 2 also needs U^n of this thread's cells in the update; their loads
  // are issued here so that the face work hides their latency
  constexpr int PASSES = G::PASSES;
  T bpre[PASSES][4];
  if (STAGE == 2) {
    const T* Bi = base + 4 * I.cell_off;
#pragma unroll
    for (int pass = 0; pass < PASSES; ++pass) {
      const int ty = threadIdx.x / TX + pass * ROWS_PER_PASS;
      const int gx = x0 + threadIdx.x % TX, gy = y0 + ty;
      const bool in = gx < I.nx && ty < desc_rows(tl.w);
      const long long c = in ? (long long)gy * I.nx + gx : 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) bpre[pass][k] = in ? Bi[k * cells + c] : T(0);
    }
  }
  if (tma) {
    __syncthreads();  // barrier initialised, row bases stored
    tma_wait(&s_bar, run, inst);
    prim_from_box<T, G::EX, G::EY, G::EY>(box, 2, P, sRB, sW);
  }
  __syncthreads();
  for (int f = threadIdx.x; f < G::NFX + G::NFY; f += NTH) {
    T w[4][4], F[4];
    if (f < G::NFX) {  // x face fx of row fy: between tile cells fx-1 and fx
      const int fy = f / (TX + 1), fx = f - fy * (TX + 1);
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const Q4<T> c = sW[(fy + 2) * G::EX + fx + p];
#pragma unroll
        for (int q = 0; q < 4; ++q) w[p][q] = c.v[q];
      }
      face_flux<T, 0>(w, lim, P.gamma, P.gm1, fs, F);
      Q4<T> fq;
#pragma unroll
      for (int q = 0; q < 4; ++q) fq.v[q] = F[q];
      sF[f] = fq;
    } else {  // y face fy of column fx: between tile rows fy-1 and fy
      const int g = f - G::NFX;
      const int fy = g / TX, fx = g - fy * TX;
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const Q4<T> c = sW[(fy + p) * G::EX + fx + 2];
#pragma unroll
        for (int q = 0; q < 4; ++q) w[p][q] = c.v[q];
      }
      face_flux<T, 1>(w, lim, P.gamma, P.gm1, fs, F);
      Q4<T> gq;
#pragma unroll
      for (int q = 0; q < 4; ++q) gq.v[q] = F[q];
      sG[g] = gq;
    }
  }
  __syncthreads();

  const int tx = threadIdx.x % TX;
  T w = T(1e30);
  bool bad = false;
  long long badc = 0;
#pragma unroll
  for (int pass = 0; pass < PASSES; ++pass) {
    const int ty = threadIdx.x / TX + pass * ROWS_PER_PASS;
    const int gx = x0 + tx, gy = y0 + ty;
    if (gx < I.nx && ty < desc_rows(tl.w)) {
      const long long c = (long long)gy * I.nx + gx;
      const T u[4] = {Si[c], Si[cells + c], Si[2 * cells + c], Si[3 * cells + c]};
      const RowBase rb = sizeof(T) == 4 ? sRB[ty + 2] : RowBase{0.f, 0.f};
      T o[4];
      const Q4<T> fl = sF[ty * (TX + 1) + tx], fr = sF[ty * (TX + 1) + tx + 1];
      const Q4<T> gd = sG[ty * TX + tx], gu = sG[(ty + 1) * TX + tx];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        T b = u[k] + sc.dtdx * (fl.v[k] - fr.v[k]);
        b = b + sc.dtdy * (gd.v[k] - gu.v[k]);
        if (k == 2) b = b + sc.dt * (state_rho(u[0], rb) * P.g);
        if (k == 3) b = b + sc.dt * (u[2] * P.g);
        o[k] = b;
      }
      if (STAGE == 2) {
#pragma unroll
        for (int k = 0; k < 4; ++k) o[k] = T(0.5) * bpre[pass][k] + T(0.5) * o[k];
      }
      T* Di = dst + 4 * I.cell_off;
#pragma unroll
      for (int k = 0; k < 4; ++k) Di[k * cells + c] = o[k];
      if (STAGE == 2 && MODE == 0) {
        bool b = false;
        const T cw = crossing_time<T>(o[0], o[1], o[2], o[3], rb, P, b);
        if (b) { bad = true; badc = c; } else if (cw < w) w = cw;
      }
    }
  }
  if (STAGE == 2 && MODE == 0) {
    if (commit_crossing<T>(w, badc, bad, I.run_tiles_h[G::LIST], run, inst, red)) {
      const double dt = run.dtrec[(long long)inst * run.max_steps + n];
      const double t = run.t[inst];
      const double tn = I.nsteps > 0 ? t + dt : (dt >= I.T - t ? I.T : t + dt);
      run.t[inst] = tn;
      run.nstep[inst] = n + 1;
      finish_step<T>(I, run, inst, n + 1, tn);
    }
  }
  if (STAGE == 2 && MODE == 1 && x0 == 0 && y0 == 0 && threadIdx.x == 0) run.nstep[inst] = n + 1;
}

// ----------------------------------------------------------------- adjoint
// Shared memory, cell-major (the 4 values of a cell together, Q4): primitive
// tile with 3 ghost layers, cotangent tile with 2, and one face buffer (the
// 4 variables of each of the face's 4 cells) used first by the x faces and
// then by the y faces.
// Geometry of an adjoint tile of H rows (32 columns), two cells per thread:
// 16 rows on 256 threads (3 FP32 CTAs per SM) or 24 rows on 384 threads (2
// FP32 CTAs per SM: the same 24 warps, a third fewer halo faces per cell and
// block barriers per cell). Every cell sums its contributions in the same
// order in both, so both give the same values.
template <int H>
struct AdjTile {
  static_assert(H == 16 || H == 24, "adjoint tiles of 16 or 24 rows");
  static constexpr int ROWS = H;
  static constexpr int NT = H == 24 ? 384 : 256;
  static constexpr int MIN_CTAS = H == 24 ? 2 : 3;  // FP32 CTAs per SM (launch bounds)
  static constexpr int RPP = NT / TX;                // tile rows covered by one pass of the block
  static constexpr int PASSES = H / RPP;
  static constexpr int AX = TX + 6, AY = H + 6, KX = TX + 4, KY = H + 4;
  static constexpr int NFX = (TX + 3) * H, NFY = TX * (H + 3);
  static constexpr int FACES = NFX > NFY ? NFX : NFY;
  static constexpr int SMEM_ELEMS = 4 * AX * AY + 4 * KX * KY + 16 * FACES;
  static_assert(H % RPP == 0, "tile rows must be a multiple of the rows per pass");
};

template <class T, int LIM, int AH>
__global__ void __launch_bounds__(AdjTile<AH>::NT, sizeof(T) == 4 ? AdjTile<AH>::MIN_CTAS : 1)
k_adjoint(const InstDev* __restrict__ insts, const int4* __restrict__ tiles, const T* __restrict__ U,
          const T* __restrict__ K, T kscale, const T* __restrict__ E, T escale, T* __restrict__ out, RunDev run,
          int n, const __grid_constant__ TileMaps tmu, const __grid_constant__ TileMaps tmk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using G = AdjTile<AH>;
  Q4<T>* sW = reinterpret_cast<Q4<T>*>(smem_raw);  // [AY][AX]
  Q4<T>* sK = sW + G::AX * G::AY;                   // [KY][KX]
  Q4<T>* sB = sK + G::KX * G::KY;                   // [4][FACES]
  __shared__ RowBase sRB[G::AY];
  __shared__ __align__(8) uint64_t s_bar;
  const int4 tl = tiles[blockIdx.x];
  const InstDev& I = insts[tl.x];
  const int inst = desc_run(tl.w);
  const StepC<T> sc = step_const<T>(run, inst, n);
  if (!(sc.dt > T(0))) return;
  const Phys<T> P = phys<T>(I);
  const long long cells = (long long)I.nx * I.ny;
  const T* Ui = U + 4 * I.cell_off;
  const T* Ki = K + 4 * I.cell_off;
  const int x0 = tl.y, y0 = tl.z, nx = I.nx, ny = I.ny;
  const int lim = LIM >= 0 ? LIM : I.limiter;
  const FluxSel<T> fs = flux_sel<T, LIM>(I);
  constexpr int PASSES = G::PASSES;
  // state and cotangent boxes by TMA, staged in the (not yet used) face buffer
  constexpr int UBOX = 4 * G::AY * TMA_BOX_X, KBOX = 4 * G::KY * TMA_BOX_X;
  static_assert(16 * G::FACES >= UBOX + KBOX + 128 / sizeof(T), "staging area too small");
  static_assert(UBOX * sizeof(T) % 128 == 0, "the cotangent box must stay 128-byte aligned");
  const bool tma = tma_tile(I, x0, y0, G::ROWS, 3);
  T* ubox = align128<T>(sB);
  T* kbox = ubox + UBOX;
  if (tma && threadIdx.x == 0) {
    mbar_init_expect(&s_bar, (UBOX + KBOX) * sizeof(T));
    if (!run.tma_skip) {
      tma_box(ubox, &tmu.m[I.tma_g], x0 - 4, y0 - 3, I.tma_z, &s_bar);
      tma_box(kbox, &tmk.m[I.tma_g], x0 - 4, y0 - 2, I.tma_z, &s_bar);
    }
  }
  // E of this thread's cells (added at the end) is loaded first, so that the
  // face work hides its latency
  T epre[PASSES][4];
#pragma unroll
  for (int pass = 0; pass < PASSES; ++pass) {
    const int gx = x0 + threadIdx.x % TX, gy = y0 + threadIdx.x / TX + pass * G::RPP;
    const bool in = E && gx < nx && gy < ny;
    const long long c = in ? 4 * I.cell_off + (long long)gy * nx + gx : 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) epre[pass][q] = in ? E[c + q * cells] : T(0);
  }

  if (tma) {
    if (sizeof(T) == 4 && threadIdx.x < G::AY) sRB[threadIdx.x] = row_base<T>(I, y0 - 3 + threadIdx.x);
    __syncthreads();  // barrier initialised, row bases stored
    tma_wait(&s_bar, run, inst);
    prim_from_box<T, G::AX, G::AY, G::AY, G::NT>(ubox, 1, P, sRB, sW);
    constexpr int N = G::KX * G::KY, PER = (N + G::NT - 1) / G::NT, PL = G::KY * TMA_BOX_X;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int e = threadIdx.x + k * G::NT;
      if (e < N) {
        const int ey = e / G::KX, ex = e - ey * G::KX;
        const T* b = kbox + ey * TMA_BOX_X + ex + 2;
        Q4<T> kc;
#pragma unroll
        for (int q = 0; q < 4; ++q) kc.v[q] = kscale * b[q * PL];
        sK[e] = kc;
      }
    }
  } else {  // cotangent tile: all loads first (rows beyond the walls hold zero)
    constexpr int N = G::KX * G::KY, PER = (N + G::NT - 1) / G::NT;
    // tile and halo inside the grid, decided once for the CTA: direct addressing
    const bool interior = x0 >= 2 && x0 + G::KX - 2 <= nx && y0 >= 2 && y0 + G::KY - 2 <= ny;
    T kv[PER][4];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int e = threadIdx.x + k * G::NT;
      const int ey = e / G::KX, ex = e - ey * G::KX;
      const int gy = y0 + ey - 2;
      if (interior) {
        const T* p = Ki + ((long long)gy * nx + x0 + ex - 2);
#pragma unroll
        for (int q = 0; q < 4; ++q) kv[k][q] = e < N ? p[q * cells] : T(0);
      } else {
        const bool in = e < N && gy >= 0 && gy < ny;
        const long long c = in ? (long long)gy * nx + wrap_x(x0 + ex - 2, nx) : 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) kv[k][q] = in ? Ki[q * cells + c] : T(0);
      }
    }
    load_prim_tile<T, G::AX, G::AY, true, G::NT>(Ui, I, cells, x0 - 3, y0 - 3, P, reinterpret_cast<T*>(sW), sRB);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int e = threadIdx.x + k * G::NT;
      if (e < N) {
        Q4<T> kc;
#pragma unroll
        for (int q = 0; q < 4; ++q) kc.v[q] = kscale * kv[k][q];
        sK[e] = kc;
      }
    }
  }
  __syncthreads();

  const int tx = threadIdx.x % TX;
  T bW[PASSES][4];
#pragma unroll
  for (int pass = 0; pass < PASSES; ++pass)
#pragma unroll
    for (int q = 0; q < 4; ++q) bW[pass][q] = T(0);

  // x faces: fx of row fy is the left face of tile cell fx-1 (cells fx-3 .. fx)
  for (int f = threadIdx.x; f < G::NFX; f += G::NT) {
    const int fy = f / (TX + 3), fx = f - fy * (TX + 3);
    T w[4][4], mu[4], o[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const Q4<T> c = sW[(fy + 3) * G::AX + fx + p];
#pragma unroll
      for (int q = 0; q < 4; ++q) w[p][q] = c.v[q];
    }
    {
      const Q4<T> kr = sK[(fy + 2) * G::KX + fx + 1], kl = sK[(fy + 2) * G::KX + fx];
#pragma unroll
      for (int q = 0; q < 4; ++q) mu[q] = sc.dtdx * (kr.v[q] - kl.v[q]);
    }
    face_vjp<T, 0>(w, mu, lim, P.gamma, P.gm1, fs, o);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      Q4<T> c;
#pragma unroll
      for (int q = 0; q < 4; ++q) c.v[q] = o[p][q];
      sB[p * G::FACES + f] = c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int pass = 0; pass < PASSES; ++pass) {
    const int ty = threadIdx.x / TX + pass * G::RPP;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const Q4<T> c = sB[p * G::FACES + ty * (TX + 3) + tx + 3 - p];
#pragma unroll
      for (int q = 0; q < 4; ++q) bW[pass][q] += c.v[q];
    }
  }
  __syncthreads();

  // y faces: fy of column fx is the bottom face of tile row fy-1 (global face y0+fy-1)
  for (int f = threadIdx.x; f < G::NFY; f += G::NT) {
    const int fy = f / TX, fx = f - fy * TX;
    const int gf = y0 + fy - 1;
    T o[4][4];
    if (gf >= 0 && gf <= ny) {
      T w[4][4], mu[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const Q4<T> c = sW[(fy + p) * G::AX + fx + 3];
#pragma unroll
        for (int q = 0; q < 4; ++q) w[p][q] = c.v[q];
      }
      const Q4<T> ku = sK[(fy + 1) * G::KX + fx + 2], kd = sK[fy * G::KX + fx + 2];
#pragma unroll
      for (int q = 0; q < 4; ++q) mu[q] = sc.dtdy * (ku.v[q] - kd.v[q]);
      face_vjp<T, 1>(w, mu, lim, P.gamma, P.gm1, fs, o);
    } else {
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) o[p][q] = T(0);
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      Q4<T> c;
#pragma unroll
      for (int q = 0; q < 4; ++q) c.v[q] = o[p][q];
      sB[p * G::FACES + f] = c;
    }
  }
  __syncthreads();

#pragma unroll
  for (int pass = 0; pass < PASSES; ++pass) {
    const int ty = threadIdx.x / TX + pass * G::RPP;
    const int gx = x0 + tx, gy = y0 + ty;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const Q4<T> c = sB[p * G::FACES + (ty + 3 - p) * TX + tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) bW[pass][q] += c.v[q];
    }
    // ghost rows of the y boundary fold back onto the cells they mirror
    for (int side = 0; side < 2; ++side) {
      int k, gly;
      if (side == 0) { if (gy > 1) continue; k = gy; gly = -1 - k - y0; }
      else { if (gy < ny - 2 || gy >= ny) continue; k = ny - 1 - gy; gly = ny + k - y0; }
      T gq[4] = {T(0), T(0), T(0), T(0)};
      const int f_lo = gly > 0 ? gly : 0, f_hi = (gly + 3) < (G::ROWS + 2) ? (gly + 3) : (G::ROWS + 2);
      for (int fy = f_lo; fy <= f_hi; ++fy) {
        const int p = gly - fy + 3;
        const Q4<T> c = sB[p * G::FACES + fy * TX + tx];
#pragma unroll
        for (int q = 0; q < 4; ++q) gq[q] += c.v[q];
      }
      bW[pass][0] += gq[0];
      bW[pass][1] += gq[1];
      bW[pass][2] -= gq[2];
      bW[pass][3] += gq[3];
      if (I.bc_y == 1) {
        const T dyk = (T)((double)(2 * k + 1) * I.dy);
        if (side == 0) bW[pass][0] -= P.g * dyk * gq[3];
        else bW[pass][0] += P.g * dyk * gq[3];
      }
    }
    // every held row; a slab's halo rows among them are overwritten by the
    // halo exchange that follows the launch (the adjoint has no reduction)
    if (gx < nx && gy < ny) {
      const long long c = (long long)gy * nx + gx;
      // rho, u_x, u_y of the cell from the primitive tile (the values mx/rho, my/rho)
      const Q4<T> wc = sW[(ty + 3) * G::AX + tx + 3];
      const T r = wc.v[0], u = wc.v[1], v = wc.v[2];
      const T* b = bW[pass];
      T bU[4];
      bU[0] = b[0] - (u * b[1] + v * b[2]) / r + P.gm1 * T(0.5) * (u * u + v * v) * b[3];
      bU[1] = b[1] / r - P.gm1 * u * b[3];
      bU[2] = b[2] / r - P.gm1 * v * b[3];
      bU[3] = P.gm1 * b[3];
      const Q4<T> kq = sK[(ty + 2) * G::KX + tx + 2];
      T kc[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) kc[q] = kq.v[q];
      T o[4];
      o[0] = kc[0] + bU[0] + sc.dtg * kc[2];
      o[1] = kc[1] + bU[1];
      o[2] = kc[2] + bU[2] + sc.dtg * kc[3];
      o[3] = kc[3] + bU[3];
      if (E) {
#pragma unroll
        for (int q = 0; q < 4; ++q) o[q] = o[q] + escale * epre[pass][q];
      }
      T* Oi = out + 4 * I.cell_off;
#pragma unroll
      for (int q = 0; q < 4; ++q) Oi[q * cells + c] = o[q];
    }
  }
}

// ------------------------------------------- gradient through the step control
// dt_n = cfl * (min over cells and directions of d / (|u_d| + c)) of U^n, or
// T - t_n when the step was clipped to the horizon. Its derivative is shared
// equally by every (cell, direction) whose crossing time equals the recorded
// minimum; |u| has derivative sign(u) with sign(0) = 0.

// Crossing times (x, y) of one conserved state, as crossing_time() computes them.
template <class T>
__device__ __forceinline__ void crossing_pair(T s0, T s1, T s2, T s3, const InstDev& I, int row, const Phys<T>& P,
                                              T& wx, T& wy) {
  T W[4];
  state_to_prim(s0, s1, s2, s3, I, row, P.gm1, W);
  const T c = sqrt(P.gamma * W[3] / W[0]);
  wx = P.dx / (fabs(W[1]) + c);
  wy = P.dy / (fabs(W[2]) + c);
}

// Per-tile partial sums for b_n dt_n = <lam^{n+1}, dU^{n+1}/d dt_n> dt_n =
// <lam1, U1 - U^n> + <lam^{n+1}, U^{n+1} - U^n/2 - U1/2> (SSP-RK2, with
// lam1 = lam^{n+1}/2 + (d(dt L)/dU1)^T lam^{n+1}/2), and the number of
// candidates of the minimum.
template <class T>
__global__ void __launch_bounds__(NTH) k_dt_partials(const InstDev* __restrict__ insts, const int4* __restrict__ tiles,
                                                     const T* __restrict__ U, const T* __restrict__ U1,
                                                     const T* __restrict__ Un1, const T* __restrict__ lam,
                                                     const T* __restrict__ lam1, RunDev run, int n,
                                                     double* __restrict__ partials) {
  __shared__ double red[NTH / 32];
  const int4 tl = tiles[blockIdx.x];
  const InstDev& I = insts[tl.x];
  const long long k = (long long)I.run * run.max_steps + n;
  const double dt = run.dtrec[k], wmin = run.wrec[k];
  const Phys<T> P = phys<T>(I);
  const long long cells = (long long)I.nx * I.ny, off = 4 * I.cell_off;
  double s = 0.0, cnt = 0.0;
  if (dt > 0.0) {
    for (int e = threadIdx.x; e < TX * TY; e += NTH) {
      const int gx = tl.y + e % TX, gy = tl.z + e / TX;
      if (gx >= I.nx || gy >= I.own1) continue;
      const long long c = off + (long long)gy * I.nx + gx;
      T u[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        u[q] = U[c + q * cells];
        const double a = (double)U1[c + q * cells], b = (double)Un1[c + q * cells];
        s += (double)lam1[c + q * cells] * (a - (double)u[q]) +
             (double)lam[c + q * cells] * (b - 0.5 * (double)u[q] - 0.5 * a);
      }
      if (wmin > 0.0) {
        T wx, wy;
        crossing_pair<T>(u[0], u[1], u[2], u[3], I, gy, P, wx, wy);
        cnt += ((double)wx == wmin ? 1.0 : 0.0) + ((double)wy == wmin ? 1.0 : 0.0);
      }
    }
  }
  s = block_sum(s, red);
  cnt = block_sum(cnt, red);
  if (threadIdx.x == 0) {
    partials[2 * (long long)blockIdx.x] = s;
    partials[2 * (long long)blockIdx.x + 1] = cnt;
  }
}

// lam^n += coef[inst] * d(crossing time)/dU^n at every candidate of the minimum.
template <class T>
__global__ void __launch_bounds__(NTH) k_dt_apply(const InstDev* __restrict__ insts, const int4* __restrict__ tiles,
                                                  const T* __restrict__ U, T* __restrict__ lam, RunDev run, int n,
                                                  const double* __restrict__ coef) {
  const int4 tl = tiles[blockIdx.x];
  const InstDev& I = insts[tl.x];
  const long long k = (long long)I.run * run.max_steps + n;
  const double wmin = run.wrec[k], cf = coef[I.run];
  if (!(run.dtrec[k] > 0.0) || !(wmin > 0.0) || cf == 0.0) return;
  const Phys<T> P = phys<T>(I);
  const long long cells = (long long)I.nx * I.ny, off = 4 * I.cell_off;
  for (int e = threadIdx.x; e < TX * TY; e += NTH) {
    const int gx = tl.y + e % TX, gy = tl.z + e / TX;
    if (gx >= I.nx || gy >= I.own1) continue;
    const long long c = off + (long long)gy * I.nx + gx;
    const T r = U[c], mx = U[c + cells], my = U[c + 2 * cells], E = U[c + 3 * cells];
    T wx, wy;
    crossing_pair<T>(r, mx, my, E, I, gy, P, wx, wy);
    const bool hx = (double)wx == wmin, hy = (double)wy == wmin;
    if (!hx && !hy) continue;
    // w = d / (|u_d| + c): dw = -d / (|u_d| + c)^2 (sign(u_d) du_d + dc), with
    // dc = gamma / (2 c rho) (dp - (p / rho) drho), p = (gamma-1)(E - |m|^2 / (2 rho))
    double rho, p;
    state_rho_p_f64(r, mx, my, E, I, gy, rho, p);
    const double u = (double)mx / rho, v = (double)my / rho, gm1 = I.gm1;
    const double cs = sqrt(I.gamma * p / rho), q = I.gamma / (2.0 * cs * rho);
    double g[4] = {0.0, 0.0, 0.0, 0.0};
    for (int d = 0; d < 2; ++d) {
      if (d == 0 ? !hx : !hy) continue;
      const double ud = d == 0 ? u : v, s = ud > 0.0 ? 1.0 : (ud < 0.0 ? -1.0 : 0.0);
      const double a = fabs(ud), h = d == 0 ? I.dx : I.dy;
      const double K = -h / ((a + cs) * (a + cs));
      g[0] += K * (s * (-ud / rho) + q * (gm1 * 0.5 * (u * u + v * v) - p / rho));
      g[1] += K * ((d == 0 ? s / rho : 0.0) - q * gm1 * u);
      g[2] += K * ((d == 1 ? s / rho : 0.0) - q * gm1 * v);
      g[3] += K * q * gm1;
    }
#pragma unroll
    for (int qv = 0; qv < 4; ++qv) lam[c + qv * cells] = (T)((double)lam[c + qv * cells] + cf * g[qv]);
  }
}

// --------------------------------------------------------------- objective
// Final state of instance i: slot_tab[nstep[i] % tab_mod] (tab_mod 2: the
// forward ping-pong pair) or slot_tab[nstep[i]] (tab_mod 0: stored states).
// The terminal cotangent dJ/dU goes to lamA / lamB by the same parity.
template <class T>
__global__ void __launch_bounds__(NTH) k_objective(const InstDev* __restrict__ insts, const int4* __restrict__ tiles,
                                                   T* const* __restrict__ slot_tab, int tab_mod,
                                                   const int* __restrict__ nstep, double* __restrict__ ek_out,
                                                   T* lamA, T* lamB, double* __restrict__ partials) {
  __shared__ double red[NTH / 32];
  const int4 tl = tiles[blockIdx.x];
  const InstDev& I = insts[tl.x];
  const long long cells = (long long)I.nx * I.ny;
  const int ns = nstep[I.run];
  const int s = tab_mod ? (ns % tab_mod) : ns;
  const T* Si = slot_tab[s] + 4 * I.cell_off;
  double ke = 0.0, pap = 0.0;
  for (int e = threadIdx.x; e < TX * TY; e += NTH) {
    const int gx = tl.y + e % TX, gy = tl.z + e / TX;
    if (gx >= I.nx || gy >= I.own1) continue;
    const long long c = (long long)gy * I.nx + gx;
    const double r = (double)Si[c] + (sizeof(T) == 4 ? (double)I.rho0_f[gy] : 0.0);
    const double mx = (double)Si[cells + c], my = (double)Si[2 * cells + c];
    const double ek = 0.5 * (mx * mx + my * my) / r;
    const double a = ek - (I.ek0 ? I.ek0[c] : 0.0);
    ke += ek;
    pap += a * a;
    if (ek_out) ek_out[I.cell_off + c] = ek;
    if (lamA) {
      const double wgt = I.objective == 1 ? 2.0 * a * I.dA : I.dA;
      const double u = mx / r, vv = my / r;
      T* Li = ((ns & 1) ? lamB : lamA) + 4 * I.cell_off;
      Li[c] = (T)(-wgt * 0.5 * (u * u + vv * vv));
      Li[cells + c] = (T)(wgt * u);
      Li[2 * cells + c] = (T)(wgt * vv);
      Li[3 * cells + c] = T(0);
    }
  }
  const double ske = block_sum(ke, red);
  const double spap = block_sum(pap, red);
  if (threadIdx.x == 0) {
    partials[2 * (long long)blockIdx.x] = ske;
    partials[2 * (long long)blockIdx.x + 1] = spap;
  }
}

// Row sums over x for the comparison diagnostics (Sec. 4.3): sum rho and sum
// e_k = |m|^2 / (2 rho) (Eq. ke) along row y of one instance; one CTA per
// (instance, row). The instance's current state is slot_tab[nstep % 2].
template <class T>
__global__ void __launch_bounds__(NTH) k_row_sums(const InstDev* __restrict__ insts, const int2* __restrict__ rows,
                                                  T* const* __restrict__ slot_tab, const int* __restrict__ nstep,
                                                  double2* __restrict__ out) {
  __shared__ double red[NTH / 32];
  const int2 r = rows[blockIdx.x];
  const InstDev& I = insts[r.x];
  const long long cells = (long long)I.nx * I.ny;
  const T* U = slot_tab[nstep[r.x] & 1] + 4 * I.cell_off + (long long)r.y * I.nx;
  double sr = 0.0, sk = 0.0;
  for (int x = threadIdx.x; x < I.nx; x += NTH) {
    const double rho = (double)U[x] + (sizeof(T) == 4 ? (double)I.rho0_f[r.y] : 0.0);
    const double mx = U[cells + x], my = U[2 * cells + x];
    sr += rho;
    sk += 0.5 * (mx * mx + my * my) / rho;
  }
  sr = block_sum(sr, red);
  sk = block_sum(sk, red);
  if (threadIdx.x == 0) out[blockIdx.x] = make_double2(sr, sk);
}

// dJ/dv from dJ/dU0 (transpose of k_inject).
template <class T>
__global__ void __launch_bounds__(NTH) k_grad(const InstDev* __restrict__ insts, const int4* __restrict__ tiles,
                                              const T* __restrict__ lam, const double* __restrict__ v,
                                              double* __restrict__ g) {
  const int4 tl = tiles[blockIdx.x];
  const InstDev& I = insts[tl.x];
  const long long cells = (long long)I.nx * I.ny;
  const T* Li = lam + 4 * I.cell_off;
  for (int e = threadIdx.x; e < TX * TY; e += NTH) {
    const int gx = tl.y + e % TX, gy = tl.z + e / TX;
    if (gx >= I.nx || gy >= I.own1) continue;
    const long long c = (long long)gy * I.nx + gx;
    const long long vc = I.v_off + vrow(I, gy) + gx;
    const double r0 = I.rho0[gy];
    const double lE = (double)Li[3 * cells + c];
    if (I.ncomp == 2) {
      g[vc] = r0 * ((double)Li[cells + c] + v[vc] * lE);
      g[vc + I.v_plane] = r0 * ((double)Li[2 * cells + c] + v[vc + I.v_plane] * lE);
    } else {
      g[vc] = r0 * ((double)Li[2 * cells + c] + v[vc] * lE);
    }
  }
}

#ifdef RT_FIELD_KERNELS
// out[inst*width + w] = sum of partials[t*width + w] over the instance's
// tiles (times dA if scale_by_dA), summed in a fixed order. One block per
// instance.
__global__ void __launch_bounds__(NTH) k_finalize(const InstDev* __restrict__ insts, const double* __restrict__ partials,
                                                  int width, int scale_by_dA, double* __restrict__ out) {
  __shared__ double red[NTH / 32];
  const InstDev& I = insts[blockIdx.x];
  for (int wc = 0; wc < width; ++wc) {
    double s = 0.0;
    for (int t = I.tile_begin + threadIdx.x; t < I.tile_end; t += NTH) s += partials[(long long)t * width + wc];
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[blockIdx.x * width + wc] = scale_by_dA ? s * I.dA : s;
  }
}

// One sample per instance (one CTA each) from the row sums: t, total kinetic
// energy (Eq. ke) and mixing width h_mix = sum over rows of 4 f (1 - f) dy
// with f = clip((<rho>_x - rho_l) / (rho_h - rho_l), 0, 1) (Eqs. hmix,
// hmix-f), and the step count. Rows are summed in a fixed order.
__global__ void __launch_bounds__(NTH) k_series_sample(const InstDev* __restrict__ insts,
                                                       const double2* __restrict__ rowsum,
                                                       const double* __restrict__ t, const int* __restrict__ nstep,
                                                       double* __restrict__ out) {
  __shared__ double red[NTH / 32];
  const InstDev& I = insts[blockIdx.x];
  double h = 0.0, ke = 0.0;
  for (int y = threadIdx.x; y < I.ny; y += NTH) {
    const double2 s = rowsum[I.row_off + y];
    const double f = fmin(fmax((s.x / I.nx - I.rho_l) / (I.rho_h - I.rho_l), 0.0), 1.0);
    h += 4.0 * f * (1.0 - f);
    ke += s.y;
  }
  h = block_sum(h, red);
  ke = block_sum(ke, red);
  if (threadIdx.x == 0) {
    double* o = out + 4 * (long long)blockIdx.x;
    o[0] = t[blockIdx.x];
    o[1] = ke * I.dA;
    o[2] = h * I.dy;
    o[3] = (double)nstep[blockIdx.x];
  }
}

// Coefficient of the step-control term of step n, one CTA per instance:
// b = (tile partials) / dt; a clipped step stores b in blast (its dt is T
// minus the sum of the earlier ones) and adds nothing; otherwise
// coef = (b - blast) cfl / (number of candidates of the minimum).
__global__ void __launch_bounds__(NTH) k_dt_coef(const InstDev* __restrict__ insts, const double* __restrict__ partials,
                                                 RunDev run, int n, double* __restrict__ blast,
                                                 double* __restrict__ coef) {
  __shared__ double red[NTH / 32];
  const InstDev& I = insts[blockIdx.x];
  double s = 0.0, cnt = 0.0;
  for (int t = I.tile_begin + threadIdx.x; t < I.tile_end; t += NTH) {
    s += partials[2 * (long long)t];
    cnt += partials[2 * (long long)t + 1];
  }
  s = block_sum(s, red);
  cnt = block_sum(cnt, red);
  if (threadIdx.x == 0) {
    const long long k = (long long)blockIdx.x * run.max_steps + n;
    const double dt = run.dtrec[k], w = run.wrec[k];
    double cf = 0.0;
    if (dt > 0.0) {
      const double b = s / dt;
      if (w < 0.0) blast[blockIdx.x] = b;
      else if (cnt > 0.0) cf = (b - blast[blockIdx.x]) * I.cfl / cnt;
    }
    coef[blockIdx.x] = cf;
  }
}

// Per-instance maximum of per-tile partial maxima (instance = block).
__global__ void __launch_bounds__(NTH) k_finalize_max(const InstDev* __restrict__ insts,
                                                      const double* __restrict__ partials, double* __restrict__ out) {
  __shared__ double red[NTH / 32];
  const InstDev& I = insts[blockIdx.x];
  double s = 0.0;
  for (int t = I.tile_begin + threadIdx.x; t < I.tile_end; t += NTH) s = fmax(s, partials[t]);
  s = block_max(s, red);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// Per-tile partial sums over perturbation fields: MODE 0: C(a) / dA =
// sum rho0 a^2 / 2 (Eq. constraint without the cell area); MODE 1: <a, b>;
// MODE 2: max |a| (a partial maximum, not a sum).
template <int MODE>
__global__ void __launch_bounds__(NTH) k_field_reduce(const InstDev* __restrict__ insts, const int4* __restrict__ tiles,
                                                      const double* __restrict__ a, const double* __restrict__ b,
                                                      double* __restrict__ partials) {
  __shared__ double red[NTH / 32];
  const int4 tl = tiles[blockIdx.x];
  const InstDev& I = insts[tl.x];
  double s = 0.0;
  for (int e = threadIdx.x; e < TX * TY; e += NTH) {
    const int gx = tl.y + e % TX, gy = tl.z + e / TX;
    if (gx >= I.nx || gy >= I.own1) continue;
    const long long c = I.v_off + vrow(I, gy) + gx;
    for (int k = 0; k < I.ncomp; ++k) {
      const double x = a[c + k * I.v_plane];
      if (MODE == 0) s += 0.5 * I.rho0[gy] * x * x;
      else if (MODE == 1) s += x * b[c + k * I.v_plane];
      else s = fmax(s, fabs(x));
    }
  }
  s = MODE == 2 ? block_max(s, red) : block_sum(s, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// out = alpha_i a + beta_i b on perturbation fields (b may be null).
__global__ void __launch_bounds__(NTH) k_field_axpby(const InstDev* __restrict__ insts, const int4* __restrict__ tiles,
                                                     double* __restrict__ out, const double* __restrict__ alpha,
                                                     const double* __restrict__ a, const double* __restrict__ beta,
                                                     const double* __restrict__ b) {
  const int4 tl = tiles[blockIdx.x];
  const InstDev& I = insts[tl.x];
  const double al = alpha[I.run], be = beta ? beta[I.run] : 0.0;
  for (int e = threadIdx.x; e < TX * TY; e += NTH) {
    const int gx = tl.y + e % TX, gy = tl.z + e / TX;
    if (gx >= I.nx || gy >= I.own1) continue;
    const long long c = I.v_off + vrow(I, gy) + gx;
    for (int k = 0; k < I.ncomp; ++k) {
      const long long idx = c + k * I.v_plane;
      double x = al * a[idx];
      if (b) x = x + be * b[idx];
      out[idx] = x;
    }
  }
}

// out = rho0(y) dA a on perturbation fields: the gradient of the constraint
// C (Eq. constraint) at a, the normal of the budget surface. inverse != 0:
// out = a / (rho0(y) dA), the representer of the linear form a in the energy
// inner product <x, y>_E = sum rho0 x y dA that C induces.
__global__ void __launch_bounds__(NTH) k_field_weight(const InstDev* __restrict__ insts, const int4* __restrict__ tiles,
                                                      double* __restrict__ out, const double* __restrict__ a,
                                                      int inverse) {
  const int4 tl = tiles[blockIdx.x];
  const InstDev& I = insts[tl.x];
  for (int e = threadIdx.x; e < TX * TY; e += NTH) {
    const int gx = tl.y + e % TX, gy = tl.z + e / TX;
    if (gx >= I.nx || gy >= I.own1) continue;
    const long long c = I.v_off + vrow(I, gy) + gx;
    const double w = I.rho0[gy];
    for (int k = 0; k < I.ncomp; ++k) {
      const long long idx = c + k * I.v_plane;
      out[idx] = inverse ? a[idx] / (w * I.dA) : w * a[idx] * I.dA;
    }
  }
}

// Multiply each perturbation field by the interface envelope
// exp(-(y - y_int)^2 / (2 h_loc^2)) (Sec. 3.4, localised random start).
__global__ void __launch_bounds__(NTH) k_localise(const InstDev* __restrict__ insts, const int4* __restrict__ tiles,
                                                  double h_loc, double* __restrict__ v) {
  const int4 tl = tiles[blockIdx.x];
  const InstDev& I = insts[tl.x];
  for (int e = threadIdx.x; e < TX * TY; e += NTH) {
    const int gx = tl.y + e % TX, gy = tl.z + e / TX;
    if (gx >= I.nx || gy >= I.own1) continue;
    const long long c = I.v_off + vrow(I, gy) + gx;
    const double y = I.y0 + (gy + 0.5) * I.dy;
    const double d = y - I.y_int;
    const double env = exp(-(d * d) / (2.0 * h_loc * h_loc));
    for (int k = 0; k < I.ncomp; ++k) v[c + k * I.v_plane] *= env;
  }
}
#endif  // RT_FIELD_KERNELS

}  // namespace rt
