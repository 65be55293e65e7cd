// rt_internal.h -- data structures shared by the host runtime and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace rt {

// Tile of cells advanced by one CTA: TILE_X x TILE_Y cells, 256 threads.
constexpr int TILE_X = 32;
constexpr int TILE_Y = 8;
constexpr int TILE_THREADS = TILE_X * TILE_Y;

// Per-instance constants, resident on the device (one entry per instance).
// State slots hold every instance back to back: instance i's conserved plane
// k (rho, m_x, m_y, E) starts at slot + 4*cell_off + k*nx*ny, row-major with
// x fastest. Perturbation fields use the caller's layout: instance i starts
// at v + v_off, ncomp planes of nx*ny.
struct InstDev {
  int nx, ny;
  int bc_y, limiter;
  int nsteps, ncomp;
  int objective, enabled;
  long long cell_off;
  long long v_off;
  int tile_begin, tile_end;  // this instance's tiles in the tile list
  double dx, dy, dA;
  double y0, y_int;          // domain bottom and interface height
  double gamma, gm1, g_y;
  double cfl, T;
  const double* rho0;        // [ny] base density at cell centres
  const double* p0;          // [ny] base pressure at cell centres
  const double* ek0;         // [nx*ny] baseline e_k for the anomaly objective (or null)
};

// Per-run device scalars, [n_inst] each unless noted.
struct RunDev {
  double* dtrec;             // [n_inst][max_steps] dt of every step (0 = inactive)
  double* t;                 // simulated time
  int* nstep;                // steps taken
  unsigned long long* wmin;  // [2][n_inst] running min of the cell crossing time (bits of a positive double)
  int* status;               // 0 ok; 1 non-finite / non-positive state seen
  long long* bad_cell;       // first bad cell (j*nx+i)
  int max_steps;
  int n_inst;
};

}  // namespace rt
