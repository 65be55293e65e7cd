// rt_internal.h -- data structures shared by the host runtime and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace rt {

// Tile of cells advanced by one CTA of the tile kernels: TILE_X x TILE_Y
// cells, 256 threads, two cells per thread (the stage kernel also has tiles of
// 8 and 32 rows, the FP32 adjoint of 24 rows on 384 threads).
constexpr int TILE_X = 32;
constexpr int TILE_Y = 16;
constexpr int TILE_THREADS = 256;

// Strip of cells advanced by one warp of the sweep kernels: STRIP_W useful
// columns (the warp's 32 lanes also cover 2 halo columns on each side) by
// STRIP_H rows, marched row by row. STRIP_WARPS strips per CTA.
constexpr int STRIP_W = 28;
constexpr int STRIP_H = 16;
constexpr int STRIP_WARPS = 4;

// Stage-kernel variants (same values bit for bit, different schedules): the
// warp sweep, and the shared-memory tile kernel with tiles of 16, 8 or 32
// rows (32 columns). Every variant has its own work list of tiles.
enum { STAGE_SWEEP = 1, STAGE_TILE = 2, STAGE_TILE8 = 3, STAGE_TILE32 = 4 };
constexpr int tile_rows_of(int variant) { return variant == STAGE_TILE8 ? 8 : (variant == STAGE_TILE32 ? 32 : 16); }
constexpr int tile_list_of(int variant) { return variant == STAGE_TILE8 ? 0 : (variant == STAGE_TILE32 ? 2 : 1); }

// Tensor-memory-accelerator (TMA) tile loads. A TMA group is a run of
// consecutive device instances of one grid shape; over a state slot it is the
// 4-D tensor (x, y, component, instance) with x fastest, described by one
// tensor map per slot and group. A launch passes the maps of the slots it
// reads; instances outside every group (and tiles whose box would leave the
// grid) use plain loads. The box spans TMA_BOX_X columns from x0 - 4 (16-byte
// aligned, since x0 is a multiple of 32), the tile's rows with their ghost
// rows, and the 4 components of one instance.
constexpr int TMA_GROUPS = 4;
constexpr int TMA_BOX_X = TILE_X + 8;
struct TileMaps {
  CUtensorMap m[TMA_GROUPS];
};

// Per-instance constants, resident on the device (one entry per device
// instance). State slots hold every device instance back to back: instance
// i's conserved plane k (rho, m_x, m_y, E) starts at slot + 4*cell_off +
// k*nx*ny, row-major with x fastest. Perturbation fields use the caller's
// layout: the cell (gy, gx) of component k is v[v_off + k*v_plane +
// (gy - own0)*nx + gx].
//
// A problem split into y-slabs has one device instance per slab: ny rows
// held (its owned rows plus halo rows copied from the neighbouring slabs
// before every kernel that reads them), own0 the first owned row, and the
// problem's index `run`, which selects the per-problem time-step control and
// scalars that all its slabs share (the tile and strip descriptors carry it
// too, with their row count). Kernels compute owned rows only and read
// halo rows as interior data. Without slabs run is the instance's own index,
// own0 = 0, own1 = ny and v_plane = nx*ny.
struct InstDev {
  int nx, ny;
  int run;                   // problem index: run scalars, dt record, per-problem coefficients
  int run_tiles, run_strips; // tiles / strips of the whole problem (all its slabs)
  int run_tiles_h[3];        // the problem's tiles in the tile-stage lists of 8, 16 and 32 rows
  int own0, own1;            // owned rows [own0, own1); the rest are halo rows
  int tma_g, tma_z;          // TMA group (-1: plain loads only) and index within it
  long long v_plane;         // stride between perturbation components
  int bc_y, limiter;
  int nsteps, ncomp;
  int objective, enabled;
  long long cell_off;
  long long v_off;
  int tile_begin, tile_end;  // this instance's tiles in the tile list
  int strip_begin, strip_end;  // this instance's strips in the sweep list
  double dx, dy, dA;
  double y0, y_int;          // domain bottom and interface height
  double rho_l, rho_h;       // light and heavy densities (mixing width, Eq. hmix-f)
  long long row_off;         // first row of this instance in the all-instance row list
  double gamma, gm1, g_y;
  double cfl, T;
  float gamma_f, gm1_f, g_f, dx_f, dy_f;  // the same constants rounded once for FP32 kernels
  int flux;                  // RT_FLUX_HLLC | RT_FLUX_HLL | RT_FLUX_HYBRID
  double flux_theta;         // hybrid threshold on the face pressure ratio (0 unless hybrid)
  float flux_theta_f;
  const double* rho0;        // [ny] base density at cell centres
  const double* p0;          // [ny] base pressure at cell centres
  // [ny] rho0 and p0 rounded to FP32. An FP32 state stores the deviation of
  // each cell from its row's base (rho0, 0, 0, p0/(gamma-1)); the kernels add
  // these back wherever they need the full state.
  const float* rho0_f;
  const float* p0_f;
  const double* ek0;         // [nx*ny] baseline e_k for the anomaly objective (or null)
};

// Per-run device scalars, [n_inst] each unless noted. The time-step control
// of step n+1 is computed once per instance by the last CTA of step n's
// stage-2 launch (or of the inject launch for step 0), which writes dt in
// FP64 (dtrec) and the per-step constants in the state precision (dtc).
struct RunDev {
  double* dtrec;             // [n_inst][max_steps] dt of every step (0 = inactive)
  double* wrec;              // [n_inst][max_steps] min crossing time behind dt (-1: step clipped to T; 0: inactive)
  void* dtc;                 // [n_inst][max_steps] StepC<T>: dt, dt/dx, dt/dy, dt*g_y in T
  double* t;                 // simulated time
  int* nstep;                // steps taken
  unsigned long long* wmin;  // running min of the cell crossing time (bits of a positive double)
  unsigned int* counter;     // CTAs of the instance finished in the current launch
  int* status;               // 0 ok; 1 non-finite / non-positive state seen; 2 a TMA tile load timed out
  long long* bad_cell;       // first bad cell (j*nx+i)
  int max_steps;
  int n_inst;
  int tma_polls = 1 << 18;   // bound on the polls of a TMA wait (see tma_wait)
  int tma_skip = 0;          // fault injection: barriers armed, no copy issued, so every TMA wait runs out
};

template <class T>
struct StepC {
  T dt, dtdx, dtdy, dtg;
};

}  // namespace rt
