/* rt_cnop.h -- C ABI of the B300 library for conditional nonlinear optimal
 * perturbations (CNOP) of the 2D compressible Rayleigh-Taylor instability.
 *
 * The paper (arXiv 2608.04085) defines the problem this library solves:
 *   * Sec. 2.1, Eqs. mass/momentum/energy and total_energy: 2D compressible
 *     Euler equations with a uniform gravity source, ideal-gas EOS;
 *   * Sec. 2.1-2.2, Eq. rho0: periodic x; tanh density interface in
 *     hydrostatic balance; y boundary reflecting or hydrostatic;
 *   * Sec. 2.3: finite-volume Godunov scheme with "hybrid HLLC" fluxes and a
 *     gravity source (this library: PLM on primitive variables, HLLC with
 *     Davis wave speeds by default, or HLL, or an HLLC/HLL hybrid switched by
 *     the face pressure ratio (rt_problem.flux); SSP-RK2, CFL time step);
 *   * Sec. 3.1, Eqs. ke, objective, constraint: the forward map F_t from a
 *     velocity perturbation v0, the objective J (final kinetic energy, or the
 *     squared kinetic-energy-density anomaly) and the budget C(v0) <= eps;
 *   * Sec. 3.4, Eq. projection: exact discrete gradient dJ/dv0 by reverse
 *     mode with checkpointing, projection P onto the budget, and a projected
 *     gradient maximisation with a non-monotone Armijo line search.
 *
 * Conventions shared by every call:
 *   * Every call returns rt_status; no C++ exception crosses the ABI. On
 *     failure rt_last_error(ctx) returns a message owned by the context.
 *   * A context owns all device memory (states, checkpoints, dt records) and
 *     a CUDA stream of its own; each call first orders that stream after the
 *     stream given to rt_init (NULL = legacy default stream), so device
 *     inputs produced there are complete before they are read. Calls are
 *     synchronous with respect to the host: they return after their device
 *     work has finished. The time loop and the checkpoint segments of the
 *     reverse sweep run as CUDA graphs captured on first use and replayed
 *     from a per-context cache (environment RT_CNOP_GRAPHS=0 disables them).
 *   * Other environment switches, read by rt_init: RT_CNOP_ADJ_ROWS=16|24
 *     fixes the FP32 adjoint's tile height (rt_adjoint_rows), and
 *     RT_CNOP_TMA_WAIT_FAULT=1 is fault injection for tests: the tile kernels
 *     arm their TMA barriers without issuing a copy, so every call that runs
 *     them ends with RT_ETIMEOUT (nothing is left in flight).
 *   * Perturbations and gradients are FP64, layout [instance][component][ny][nx]
 *     (C-contiguous, x fastest); instances are concatenated in order, each
 *     with perturb_ncomp components (1: u_y only; 2: u_x then u_y).
 *     rt_field_offset / rt_field_size give each instance's place.
 *   * Pointer arguments are host pointers unless RT_DEVICE_PTRS is set in
 *     `flags`, in which case the perturbation / gradient arrays are device
 *     pointers on the context's device (e.g. torch.Tensor.data_ptr()).
 *     Scalar outputs (J, C, statistics) are always host arrays.
 *   * The caller owns every array it passes; the library keeps no pointer to
 *     caller memory after a call returns.
 *
 * A typical sequence (host arrays, one FP32 batch, error checks elided):
 *
 *   rt_problem p[32];  ... fill each instance ...
 *   rt_options o = {RT_FP32_STATE, RT_CKPT_AUTO, 0.0, 0, RT_STAGE_AUTO, 0, RT_LOADS_TMA};
 *   rt_ctx* ctx;
 *   rt_init(p, 32, &o, NULL, &ctx);
 *   size_t n = rt_field_total(ctx);              // doubles in v0 and grad
 *   double J[32], *v0 = ..., *grad = ...;         // v0: seeded N(0,1) fields
 *   double eps[32] = {1e-4, ...};
 *   rt_project(ctx, v0, 0, eps, 1);               // scale onto C = eps
 *   rt_gradient(ctx, v0, 0, J, grad, NULL);       // J and dJ/dv0
 *   cnop_params cp = {0};                         // zero fields take their defaults,
 *   cp.max_iter = 50;  cp.armijo_c = 1e-4;        // except armijo_c (0 = no sufficient increase)
 *   cp.eps = eps;  cp.method = RT_CNOP_LBFGS;
 *   cnop_result cr = {0};
 *   cnop_solve(ctx, &cp, v0, 0, J, &cr);          // v0 becomes the CNOP
 *   rt_destroy(ctx);
 */
#ifndef RT_CNOP_H
#define RT_CNOP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rt_ctx rt_ctx;

typedef enum {
  RT_OK = 0,
  RT_EINVAL = 1,        /* bad argument, shape or parameter */
  RT_ENOMEM = 2,        /* device or host allocation failed */
  RT_ECUDA = 3,         /* a CUDA runtime call failed */
  RT_ENONFINITE = 4,    /* non-positive density/pressure or NaN in a state */
  RT_ETIMEOUT = 5,      /* a bounded device wait gave up */
  RT_ENOTCONVERGED = 6, /* optimiser stopped without an accepted step */
  RT_ESTATE = 7,        /* call out of order (e.g. replay before any run) */
  RT_EIO = 8            /* reading or writing a file failed */
} rt_status;

enum { RT_BC_REFLECT = 0, RT_BC_HYDROSTATIC = 1 };
enum { RT_LIM_MINMOD = 0, RT_LIM_MC = 1, RT_LIM_NONE = 2 };
enum { RT_FLUX_HLLC = 0, RT_FLUX_HLL = 1, RT_FLUX_HYBRID = 2 };
enum { RT_OBJ_KE = 0, RT_OBJ_EK_ANOMALY_L2 = 1 };
enum { RT_FP64 = 0, RT_FP32_STATE = 1 };
enum { RT_CKPT_AUTO = 0, RT_CKPT_STORE_ALL = 1, RT_CKPT_SQRT = 2, RT_CKPT_REVOLVE = 3 };
enum { RT_STAGE_AUTO = 0, RT_STAGE_SWEEP = 1, RT_STAGE_TILE = 2, RT_STAGE_TILE8 = 3, RT_STAGE_TILE32 = 4 };
/* rt_options.tile_loads */
enum { RT_LOADS_TMA = 0, RT_LOADS_PLAIN = 1 };
enum { RT_CNOP_SPG = 0, RT_CNOP_LBFGS = 1 };

/* flags for rt_forward / rt_gradient / rt_constraint / rt_project / cnop_solve:
 * RT_DEVICE_PTRS  the v / grad / out pointers are device pointers;
 * RT_REPLAY_DT    rt_forward replays the previous run's dt sequence;
 * RT_GRAD_DT      rt_gradient (and cnop_solve's gradients) also differentiate
 *                 the step control, see rt_gradient. */
enum { RT_DEVICE_PTRS = 1, RT_REPLAY_DT = 2, RT_GRAD_DT = 4 };

/* One RT problem (Sec. 2.1-2.3). Geometry: cells are (x1-x0)/nx by
 * (y1-y0)/ny. Base state: rho0(y) = (rho_heavy+rho_light)/2 +
 * (rho_heavy-rho_light)/2 tanh((y-y_int)/h_s) and p0 from dp/dy = rho0 g_y
 * with p0(y_ref) = p_ref. g_y is the signed acceleration (paper -1, negative
 * = downward). nsteps > 0 runs that many CFL steps; otherwise the run ends
 * at time T, the last step clipped to T - t. */
typedef struct {
  int nx, ny;
  double x0, x1, y0, y1;
  double gamma, g_y;
  double rho_heavy, rho_light, y_int, h_s;
  double p_ref, y_ref;
  int bc_y;          /* RT_BC_REFLECT | RT_BC_HYDROSTATIC */
  int limiter;       /* RT_LIM_MINMOD | RT_LIM_MC | RT_LIM_NONE */
  double cfl;
  double T;
  int nsteps;
  int perturb_ncomp; /* 1: u_y only (Sec. 3.1); 2: (u_x, u_y) */
  int objective;     /* RT_OBJ_KE | RT_OBJ_EK_ANOMALY_L2 */
  int flux;          /* Riemann flux (Sec. 2.3, "hybrid HLLC"): RT_FLUX_HLLC (HLLC with
                        Davis speeds), RT_FLUX_HLL (HLL, same speeds) or RT_FLUX_HYBRID:
                        HLL at faces whose reconstructed pressures differ by more than
                        the factor flux_theta (p_L > flux_theta p_R or p_R > flux_theta
                        p_L), HLLC elsewhere */
  double flux_theta; /* RT_FLUX_HYBRID threshold, >= 1; ignored otherwise */
} rt_problem;

typedef struct {
  int precision;            /* RT_FP64, or RT_FP32_STATE: FP32 state with FP64 reductions.
                               The FP32 state holds each cell's deviation from the
                               hydrostatic base state of its row, so that its rounding is
                               relative to the perturbation, not to the O(1) background */
  int ckpt;                 /* RT_CKPT_AUTO | RT_CKPT_STORE_ALL | RT_CKPT_SQRT | RT_CKPT_REVOLVE;
                               AUTO takes the first that fits the cap in that order */
  double ckpt_hbm_cap_bytes;/* cap on checkpoint + segment memory; 0 = 60% of free memory.
                               REVOLVE uses cap / slot size - 4 binomial checkpoint slots */
  int max_steps;            /* upper bound on steps per run (sizes the dt record); 0 = 200000 */
  int stage_kernel;         /* RT_STAGE_AUTO (time the four variants at rt_init, keep the
                               fastest), RT_STAGE_SWEEP, RT_STAGE_TILE, RT_STAGE_TILE8 or
                               RT_STAGE_TILE32; all give the same values (FP64 bit for bit) */
  int y_slabs;              /* 0 or 1: each problem is one device instance. k > 1: each
                               problem is split into k y-slabs of nearly equal height
                               (at least 3 rows each, so ny >= 3k), each holding its rows
                               plus 3 halo rows per neighbouring slab, refreshed by
                               device-to-device copies after every kernel that writes a
                               state or a cotangent; the slabs of a problem share one time
                               step (minimum over all their cells) and every sum (J, C,
                               dot products) runs over all of them. Results equal the
                               unsplit run: state, dt sequence and gradient bit for bit,
                               sums to rounding order. rt_forward_series is not
                               available on a split context (RT_EINVAL) */
  int tile_loads;           /* RT_LOADS_TMA (default): the tile kernels fetch every tile
                               whose box lies inside the grid with one TMA tensor copy per
                               state slot (instances in runs of one shape, at most 4 runs,
                               with rows of a 16-byte multiple); other tiles use plain loads.
                               RT_LOADS_PLAIN: plain loads everywhere. Same values either
                               way. A TMA wait that gives up (bounded) fails the call with
                               RT_ETIMEOUT */
} rt_options;

typedef struct {
  int steps;                /* largest step count over instances in the last run */
  int segments;             /* checkpoint segments of the last gradient (sqrt: > 1;
                               store-all: 1; revolve: minus the recomputed steps) */
  int bad_instance;         /* RT_ENONFINITE: first instance with a non-finite or
                               non-positive state; RT_ETIMEOUT: the instance whose tile
                               load gave up; else -1 */
  int bad_step;             /* RT_ENONFINITE: the step (from 0) whose result was bad, else -1 */
  long long bad_cell;       /* RT_ENONFINITE: its first bad cell (j*nx + i), else -1. On a
                               failed rt_forward / rt_gradient only these three fields are
                               set (the others are zero) */
  double cell_updates;      /* sum over instances of cells x steps advanced */
  double ms;                /* device time of the call, CUDA events on the stream */
  long long launches;       /* kernels launched by the call */
} rt_run_stats;

/* Create a context for n_instances problems (instances may differ in grid
 * and physics but share precision and checkpoint policy). Builds the base
 * state of every instance (Sec. 2.2) on the host in FP64, uploads it, and,
 * for instances using RT_OBJ_EK_ANOMALY_L2, runs the unperturbed baseline
 * (Eq. objective) once. cuda_stream is a cudaStream_t or NULL.
 * Errors: RT_EINVAL (nx < 4, ny < 2, non-positive densities/pressures,
 * unknown enums), RT_ENOMEM, RT_ECUDA. *out is NULL on failure. */
rt_status rt_init(const rt_problem* problems, int n_instances, const rt_options* opt,
                  void* cuda_stream, rt_ctx** out);

/* Release every device buffer of the context. NULL is ignored. */
void rt_destroy(rt_ctx* ctx);

/* Message of the last failed call on this context ("" if none). */
const char* rt_last_error(const rt_ctx* ctx);

/* Number of instances, and the offset / length (in doubles) of instance i's
 * perturbation field inside the concatenated layout. */
int rt_num_instances(const rt_ctx* ctx);
size_t rt_field_offset(const rt_ctx* ctx, int inst);
size_t rt_field_size(const rt_ctx* ctx, int inst);
size_t rt_field_total(const rt_ctx* ctx);

/* Forward map F_t (Sec. 3.1): inject v0 into the base state, march every
 * instance to its horizon, and write J_out[i] = J of instance i (its
 * `objective`); J_ke_out[i] (nullable) = final total kinetic energy.
 * RT_REPLAY_DT re-uses the dt sequence recorded by the previous run instead
 * of the CFL control (frozen-dt finite differences). st is nullable.
 * Errors: RT_EINVAL, RT_ESTATE (replay without a previous run),
 * RT_ENONFINITE (st->bad_* says where), RT_ECUDA. */
rt_status rt_forward(rt_ctx* ctx, const double* v0, int flags, double* J_out,
                     double* J_ke_out, rt_run_stats* st);

/* Comparison diagnostics of one forward run (Sec. 4.3, Figs. ek_growth and
 * mixing_width): for every instance, samples of the time t, the total kinetic
 * energy KE(t) = sum e_k dx dy (Eq. ke) and the mixing width
 * h_mix(t) = sum over rows of 4 f (1 - f) dy with
 * f = clip((<rho>_x - rho_light) / (rho_heavy - rho_light), 0, 1)
 * (Eqs. hmix, hmix-f), taken at step 0, every `every` steps, and at the
 * instance's last step. Outputs are [n_instances][max_samples] row-major
 * (instance i's samples start at i * max_samples); n_out[i] = samples
 * written (samples beyond max_samples are dropped). flags as rt_forward; the
 * run counts as the previous run for RT_REPLAY_DT.
 * Errors: RT_EINVAL (null output, every < 1, max_samples < 1), as rt_forward. */
rt_status rt_forward_series(rt_ctx* ctx, const double* v0, int flags, int every, int max_samples,
                            double* t_out, double* ke_out, double* hmix_out, int* n_out);

/* Exact discrete gradient dJ/dv0 (Sec. 3.4) of the same map, dt sequence
 * frozen at the one the forward pass chose, by a hand-written adjoint of the
 * time stepper with store-all, sqrt(N) or binomial (revolve) checkpointing
 * (Sec. 3.4 uses binomial checkpointing). grad_out has the layout of v0.
 * With RT_GRAD_DT the step control is differentiated as well, as an automatic
 * differentiation of the whole forward run would do: dt_n = cfl * (min over
 * cells and directions of d / (|u_d| + c)) of U^n, its derivative shared
 * equally by every (cell, direction) equal to the minimum (|u| has derivative
 * sign(u), sign(0) = 0), and a horizon-clipped last step dt = T - t passes
 * its sensitivity to every earlier dt. This costs one extra stage and three
 * light launches per reverse step. RT_REPLAY_DT is not accepted.
 * Errors as rt_forward. */
rt_status rt_gradient(rt_ctx* ctx, const double* v0, int flags, double* J_out,
                      double* grad_out, rt_run_stats* st);

/* Eq. constraint: C_out[i] = sum over cells and components of
 * rho0 v^2 / 2 dx dy for instance i. */
rt_status rt_constraint(rt_ctx* ctx, const double* v, int flags, double* C_out);

/* Eq. projection, in place: v_i <- v_i * min(1, sqrt(eps_i / C(v_i)));
 * with to_budget != 0, v_i <- v_i * sqrt(eps_i / C(v_i)) (scale onto the
 * sphere C = eps). eps has one entry per instance. */
rt_status rt_project(rt_ctx* ctx, double* v, int flags, const double* eps, int to_budget);

/* Final conserved state (rho, m_x, m_y, E) of instance i after the last
 * forward run, as FP64 [4][ny][nx] into a host array (for an FP32 state, the
 * stored deviation plus the FP32-rounded base state, summed in FP64). */
rt_status rt_get_state(rt_ctx* ctx, int inst, double* out);

/* dt sequence of instance i recorded by the last run; *n_out = its length.
 * At most max_n values are written. */
rt_status rt_get_dt(rt_ctx* ctx, int inst, double* out, int max_n, int* n_out);

/* Kernel timing (no counterpart in the paper; measurement support). With
 * every > 0, each later call records CUDA events around every `every`-th
 * launch of the three time-step kernels on the context's stream; 0 turns
 * it off. rt_kernel_times returns, for the kernels of the last call indexed
 * 0 = stage 1, 1 = stage 2, 2 = adjoint stage: mean device time per sampled
 * launch (ms), number of samples, and number of launches (any array may be
 * NULL). */
rt_status rt_set_kernel_timing(rt_ctx* ctx, int every);

/* Stage-kernel variant in use (no counterpart in the paper): RT_STAGE_SWEEP
 * (one warp per 28 x 16 strip) or the shared-memory tile kernel with tiles
 * of 32 columns by 16 (RT_STAGE_TILE), 8 (RT_STAGE_TILE8) or 32
 * (RT_STAGE_TILE32) rows; all give the same values bit for bit in FP64.
 * With RT_STAGE_AUTO, rt_init timed four CFL steps of the unperturbed batch
 * with each of the four and kept the fastest; tuned_ms (nullable, [2])
 * receives the mean times per step of the sweep and of the 16-row tile
 * kernel, or zeros when the variant was fixed by the options. */
int rt_stage_kernel(const rt_ctx* ctx, double* tuned_ms);

/* All four autotuner timings, ms per step (no counterpart in the paper):
 * ms[0] sweep, ms[1] tiles of 8 rows, ms[2] of 16 rows, ms[3] of 32 rows;
 * zeros when the variant was fixed by the options. Errors: RT_EINVAL. */
rt_status rt_stage_tuning(const rt_ctx* ctx, double* ms);

/* Adjoint tile height in use (no counterpart in the paper): 16 (tiles of
 * 32 x 16 cells on 256 threads), or 24 (32 x 24 cells on 384 threads, FP32
 * state only); both give the same values. For FP32, rt_init timed three
 * adjoint launches of the unperturbed batch with each and kept the faster;
 * ms (nullable, [2]) receives those times per launch (zeros for FP64, which
 * always uses 16). The environment variable RT_CNOP_ADJ_ROWS=16|24 fixes the
 * choice at rt_init. Returns 0 for a null context. */
int rt_adjoint_rows(const rt_ctx* ctx, double* ms);
rt_status rt_kernel_times(rt_ctx* ctx, double* mean_ms, long long* samples, long long* launches);

typedef struct {
  int max_iter;          /* total iterations (a resumed run continues up to it) */
  int gll_memory;        /* non-monotone memory M (the reference is the smallest of the
                            last M accepted J values); 0 = 10 */
  int max_backtracks;    /* per iteration; 0 = 30 */
  double armijo_c;       /* sufficient-increase constant, e.g. 1e-4 */
  double alpha_min, alpha_max; /* SPG step safeguards; 0 = 1e-30, 1e30 */
  double h_loc;          /* > 0: multiply v_inout by exp(-(y-y_int)^2/(2 h_loc^2)) first */
  const double* eps;     /* budget per instance */
  int method;            /* RT_CNOP_SPG or RT_CNOP_LBFGS */
  int lbfgs_memory;      /* L-BFGS: pairs of the last m iterations; 0 = 10 (Sec. 3.4) */
  double chi_tol;        /* > 0: an instance stops once chi <= chi_tol (App. A) */
  const char* log_path;  /* nullable: one text line per instance and iteration
                            (iter instance J C chi grad_norm lambda forward_evals
                            gradient_evals); truncated on a fresh start, appended on resume */
  const char* checkpoint_path; /* nullable: the whole optimiser state (iterate, gradient,
                            L-BFGS pairs, step and J histories) is written here every
                            checkpoint_every iterations and on return */
  int checkpoint_every;  /* 0 = only on return */
  int resume;            /* nonzero: continue from checkpoint_path if that file exists
                            (v_inout and h_loc are then ignored) */
} cnop_params;

typedef struct {
  int iterations;        /* iterations run, counting those before a resume (lockstep batch) */
  int forward_evals;     /* batched forward runs (line-search trials) */
  int gradient_evals;    /* batched gradient runs */
  double ms;             /* device time of the whole solve */
  /* Per-instance outputs: caller-owned arrays, each NULL or n_instances long
   * (J_history: (max_iter + 1) * n_instances, row k = J after k iterations,
   * rows after the last iteration left untouched). Zero the struct, then set
   * the ones wanted. */
  double* C;             /* C of the returned iterate (Eq. constraint) */
  double* chi;           /* chi = ||P(v + dJ/dv) - v||_inf at the returned iterate (App. A) */
  double* grad_norm;     /* ||dJ/dv||_2 there */
  int* stop;             /* 0 iteration limit, 1 no acceptable step, 2 chi <= chi_tol */
  double* J_history;
} cnop_result;

/* CNOP search (Sec. 3.4, Eq. projection). Every instance starts from
 * v_inout (a seeded random field; optionally localised by h_loc), scaled onto
 * C = eps (a start with C = 0 is RT_EINVAL), and all instances advance in
 * lockstep through batched forward and gradient runs; an instance that has
 * stopped is switched off in those runs. Two methods:
 *  RT_CNOP_LBFGS (the paper's): on the budget surface C = eps the model
 *    gradient is that of J o P, gh = g - (<g,v>/<n,v>) n with n = dC/dv, and
 *    the direction is made tangent, p <- p - (<n,p>/<n,n>) n (off the surface
 *    gh = g). p = H gh from the two-loop recursion over the (s, y) pairs of
 *    the last lbfgs_memory iterations, y = -(gh_new - gh_old), a pair with
 *    <s, y> <= 0 skipped, H0 = <s, y>/<y, y> of the newest stored pair
 *    (||v||/||gh|| when none); if <gh, p> <= 0 the pairs are dropped and
 *    p = (||v||/||gh||) gh; trial points P(v + lam p), lam = 1, 1/2, ...,
 *    accepted once J >= min(last gll_memory J) + armijo_c <gh, P(v + lam p) - v>.
 *  RT_CNOP_SPG: steps in the energy inner product <a,b>_E = sum rho0 a b dA
 *    of Eq. constraint, in which P is the exact projection onto the ball, so
 *    that its fixed points are the KKT points g = lambda dC/dv: with
 *    q = g / (rho0 dA) the representer of g, d = P(v + alpha q) - v, trial
 *    points v + lam d accepted once J >= min(last gll_memory J) +
 *    armijo_c lam <g, d>, and the Barzilai-Borwein step
 *    alpha = <s,s>_E / <s,y> clipped to [alpha_min, alpha_max] (alpha_max
 *    when <s,y> <= 0); the first alpha is ||v||_E / ||q||_E.
 * On return v_inout holds the CNOP of every instance and J_out[i] (nullable)
 * its objective. Errors: as rt_gradient; RT_EINVAL for an unknown method, or
 * a checkpoint written for another context, method, memory, precision or
 * eps; RT_EIO when the log or checkpoint cannot be written or read;
 * RT_ENOTCONVERGED when an instance found no acceptable step within
 * max_backtracks trials (its last accepted iterate is returned). */
rt_status cnop_solve(rt_ctx* ctx, const cnop_params* prm, double* v_inout, int flags,
                     double* J_out, cnop_result* res);

/* Fourier analysis of perturbation fields and the reduced seeds built from
 * it (Sec. 3.5, Sec. 4.2 Eq. fourier_coeff, App. B). v has the layout of v0
 * (RT_DEVICE_PTRS: device pointer); the spectra are taken of u_y, the last
 * perturbed component of an instance. Plain DFTs with exactly reduced
 * phases, FP64; nx and ny at most 6144. E_out is a host array.
 *
 * rt_spectrum_x: y_peak = the row where the rms of u_y along x is largest
 *   (ties: lowest row); u_n = sum_j u_y(x_j, y_peak) exp(-2 pi i n j / nx) and
 *   E_out[n - 1] = |u_n|^2 / sum_m |u_m|^2 for n, m = 1 .. nx/2.
 * rt_spectrum_2d: E_out[ky * nx + kx] = |F|^2 / sum |F|^2 over all modes,
 *   F the two-dimensional DFT of u_y over the whole grid.
 * rt_reconstruct: the reduced seed of every instance, rescaled to
 *   C = eps[i] and written to out (layout of v0):
 *   RT_RECON_X_MODES, param = count: the `count` horizontal modes n with the
 *     largest E_n at y_peak (ties: lower n), with their mirrors -n, kept in
 *     every row and component (the paper's five-mode seed, count = 5);
 *   RT_RECON_2D_POWER, param = fraction in (0, 1]: the two-dimensional modes,
 *     ranked in conjugate pairs by the pair's energy, that hold `fraction`
 *     of the energy (the last pair's ties included), kept in every
 *     component (the paper's 90%-power seed, fraction = 0.9).
 *   kept_out[i] (nullable) = modes kept.
 * Errors: RT_EINVAL (bad instance, kind, parameter or size; a
 * reconstruction with C = 0), RT_ECUDA. */
enum { RT_RECON_X_MODES = 0, RT_RECON_2D_POWER = 1 };
rt_status rt_spectrum_x(rt_ctx* ctx, const double* v, int flags, int inst, double* E_out, int* y_peak_out);
rt_status rt_spectrum_2d(rt_ctx* ctx, const double* v, int flags, int inst, double* E_out);
rt_status rt_reconstruct(rt_ctx* ctx, const double* v, int flags, int kind, double param, const double* eps,
                         double* out, int* kept_out);

/* Binomial checkpoint plan (Sec. 3.4 names checkpointing; the schedule is
 * Griewank & Walther's revolve): the forward steps that rt_gradient with
 * RT_CKPT_REVOLVE recomputes to reverse `steps` time steps with `slots` free
 * checkpoint slots besides the initial state (slots = cap / slot size - 4),
 * and Griewank & Walther's minimum t n - beta(slots + 2, t - 1) with
 * beta(c, t) = C(c + t, c) and t the smallest integer with
 * beta(slots + 1, t) >= n. The two are equal: the schedule is optimal. A
 * host computation; it needs no device and no context.
 *   recomputed  host long long, the schedule's count (NULL: not written);
 *   optimum     host double, the closed-form minimum (NULL: not written).
 * Errors: RT_EINVAL (steps < 0 or slots < 0). */
rt_status rt_revolve_plan(int steps, int slots, long long* recomputed, double* optimum);

/* The TMA tile-load plan (no counterpart in the paper; host arithmetic only,
 * no device needed): for n device instances of grids nx[i] x ny[i] in slot
 * order (without y-slabs, the problems in rt_init's order) and an element
 * size of 4 (FP32 state) or 8 (FP64), which instances the tile kernels fetch
 * with TMA tensor copies. group_of[i] (host, [n]) receives the instance's
 * group, or -1 for plain loads; index_of[i] (host, [n]) its index within the
 * group. A group is a maximal run of consecutive instances of one shape
 * whose rows are a multiple of 16 bytes and whose grid holds every tile box
 * (nx >= 72, ny >= 36); at most 4 runs, the largest (cells times instances)
 * first, ties to the earlier run. rt_init keeps this plan when
 * rt_options.tile_loads is RT_LOADS_TMA and the driver can encode the tensor
 * maps. Errors: RT_EINVAL (null arrays, n < 0, another element size). */
rt_status rt_tma_plan(const int* nx, const int* ny, int n, int elem_bytes, int* group_of, int* index_of);

/* Measured FMA throughput of the current device (measurement support; the
 * paper has no counterpart): independent fused multiply-add chains in every
 * thread of a grid that fills every SM, FP32 and FP64, best of three timed
 * launches after a warm-up; tflops_* = 2 FLOPs per FMA / time. Runs on the
 * legacy default stream and synchronises the device. Errors: RT_EINVAL (null
 * output), RT_ECUDA. */
rt_status rt_fma_peak(double* tflops_f32, double* tflops_f64);

/* Allocation-free objective of one final state. The paper has no
 * counterpart: this exists for callers that must not let a library allocate
 * device memory (a host framework that owns all device memory through its
 * own pool with a fixed budget, or a loop that cannot afford the device-wide
 * synchronisation of cudaMalloc / cudaFree). It needs no context and calls
 * no allocating routine.
 *   p      grid and domain of the state (nx, ny, x0, x1, y0, y1 are used);
 *   state  device FP64 conserved state [4][ny][nx] (rho, m_x, m_y, E), the
 *          layout rt_get_state returns;
 *   ek0    device FP64 reference e_k [ny][nx], or NULL for zero;
 *   J      device FP64 [2]: J[0] = sum e_k dx dy (total kinetic energy),
 *          J[1] = sum (e_k - ek0)^2 dx dy.
 * The work is queued on cuda_stream (NULL = legacy default stream) and the
 * call returns without waiting for it. Per-block partial sums live in a
 * fixed 256 KiB device array inside the library, so grids above 4,194,304
 * cells return RT_EINVAL (with a message on stderr). The first call on each
 * device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current; make that first call before any stream capture. The
 * address is kept per device number for the life of the process: it does not
 * survive cudaDeviceReset (which unloads the library's device image), so
 * calling this entry point after a reset of that device is not supported. All
 * calls share the array: calls whose kernels overlap on the GPU race on it.
 * Errors: RT_EINVAL (null pointer, empty domain, size), RT_ECUDA. */
rt_status rt_objective_noalloc(const rt_problem* p, const double* state, const double* ek0, double* J,
                               void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* RT_CNOP_H */
