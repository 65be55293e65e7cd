// rt_oracle.cpp -- plain FP64 CPU oracle for the compressible Rayleigh-Taylor
// forward map, its tangent and its discrete adjoint.
//
// TEST INFRASTRUCTURE ONLY. Nothing on the product path may link, load or call
// this file. It exists so that tests, the smoke check and the CPU baseline of
// the benchmark can compare the CUDA library against an independent, slow,
// obviously correct implementation. It shares no code with the CUDA library.
//
// What it computes (paper sections in brackets):
//   * base state: tanh density profile and hydrostatic pressure   [Sec. 2.2, Eq. rho0]
//   * inject: U0 = (rho0, rho0 v, p0/(gamma-1) + rho0 |v|^2 / 2)   [Sec. 3.1; Eq. total_energy]
//   * one SSP-RK2 step of a finite-volume Godunov scheme: PLM on
//     primitive variables, HLLC fluxes (or HLL, or the HLLC/HLL hybrid
//     switched by the face pressure ratio), gravity source       [Sec. 2.1 Eqs. mass/momentum/energy; Sec. 2.3]
//   * CFL time step and horizon clipping (scheme fixed by the workload, Sec. 2.3 leaves it open)
//   * objectives: total kinetic energy, and the squared e_k anomaly  [Sec. 3.1, Eqs. ke, objective]
//   * tangent (forward-mode dual numbers) and reverse-mode gradient with the
//     time step frozen; the reverse uses local flux Jacobians obtained by
//     forward-mode dual numbers, transposed face by face             [Sec. 3.4]
//   * branch signature of a forward run (a test aid): which side of every
//     kink (limiter pick, Davis speed min/max, HLLC branch) each evaluation
//     took, so that finite differences straddling a kink can be told apart
// Built with -O2 -ffp-contract=off so that every expression rounds exactly as
// written; the evaluation order of each expression is part of the scheme
// definition (the CUDA FP64 path evaluates the same expressions).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include <omp.h>

extern "C" {
struct OParams {
  int nx, ny;
  double x0, x1, y0, y1;
  double gamma, g_y;
  double rho_h, rho_l, y_int, h_s;
  double p_ref, y_ref;
  int bc_y, limiter;
  double cfl, T;
  int nsteps, ncomp, objective;
  int flux;           // O_FLUX_HLLC | O_FLUX_HLL | O_FLUX_HYBRID
  double flux_theta;  // hybrid: HLL where one face pressure exceeds flux_theta times the other
};
}

enum { O_BC_REFLECT = 0, O_BC_HYDROSTATIC = 1 };
enum { O_LIM_MINMOD = 0, O_LIM_MC = 1, O_LIM_NONE = 2 };
enum { O_OBJ_KE = 0, O_OBJ_PAPER = 1 };
enum { O_FLUX_HLLC = 0, O_FLUX_HLL = 1, O_FLUX_HYBRID = 2 };
static const int H = 2;  // ghost layers needed by PLM

// Branch signature (o_forward_signature only): every kink decision of the
// scheme, as a small code, folded in evaluation order into a 64-bit FNV-1a
// hash. Off everywhere else; the oracle runs single-threaded.
static bool g_sig_on = false;
static unsigned long long g_sig = 0;
static long long g_sig_n = 0;
static inline void sig_add(int code) {
  if (!g_sig_on) return;
  g_sig ^= (unsigned long long)(unsigned)code;
  g_sig *= 1099511628211ull;
  ++g_sig_n;
}

// Host threads for the loops over rows (OpenMP). Every parallel loop writes
// rows or faces of its own and every sum keeps its serial order, so results
// are bitwise the same for any thread count. One thread by default (no
// thread pool is started, so processes forked later stay safe); the branch
// signature, a running hash, always runs on one thread.
static int g_threads = 1;
static inline int nthreads() { return g_sig_on ? 1 : g_threads; }
extern "C" void o_set_threads(int n) { g_threads = n < 1 ? 1 : n; }
extern "C" int o_get_threads() { return g_threads; }
extern "C" int o_num_procs() { return omp_get_num_procs(); }

// ---------------------------------------------------------------- dual numbers
template <int N> struct Dual {
  double v;
  double d[N];
  Dual() : v(0.0) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
  Dual(double x) : v(x) { for (int i = 0; i < N; ++i) d[i] = 0.0; }
};
template <int N> inline Dual<N> operator+(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v + b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <int N> inline Dual<N> operator-(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v - b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <int N> inline Dual<N> operator-(const Dual<N>& a) {
  Dual<N> r;
  r.v = -a.v;
  for (int i = 0; i < N; ++i) r.d[i] = -a.d[i];
  return r;
}
template <int N> inline Dual<N> operator*(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v * b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <int N> inline Dual<N> operator/(const Dual<N>& a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a.v / b.v;
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) / b.v;
  return r;
}
template <int N> inline Dual<N> operator*(double a, const Dual<N>& b) {
  Dual<N> r;
  r.v = a * b.v;
  for (int i = 0; i < N; ++i) r.d[i] = a * b.d[i];
  return r;
}
template <int N> inline Dual<N> operator*(const Dual<N>& a, double b) {
  Dual<N> r;
  r.v = a.v * b;
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b;
  return r;
}
template <int N> inline Dual<N> operator+(double a, const Dual<N>& b) { return Dual<N>(a) + b; }
template <int N> inline Dual<N> operator+(const Dual<N>& a, double b) { return a + Dual<N>(b); }
template <int N> inline Dual<N> operator-(double a, const Dual<N>& b) { return Dual<N>(a) - b; }
template <int N> inline Dual<N> operator-(const Dual<N>& a, double b) { return a - Dual<N>(b); }
template <int N> inline Dual<N> operator/(const Dual<N>& a, double b) { return a / Dual<N>(b); }
template <int N> inline Dual<N> operator/(double a, const Dual<N>& b) { return Dual<N>(a) / b; }
template <int N> inline Dual<N> sqrt(const Dual<N>& a) {
  Dual<N> r;
  r.v = std::sqrt(a.v);
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] / (2.0 * r.v);
  return r;
}
template <int N> inline Dual<N> fabs(const Dual<N>& a) { return a.v < 0.0 ? -a : a; }

inline double val(double x) { return x; }
template <int N> inline double val(const Dual<N>& x) { return x.v; }

// ------------------------------------------------------------------- geometry
struct Grid {
  int nx, ny;
  double dx, dy;
  explicit Grid(const OParams& P) : nx(P.nx), ny(P.ny),
      dx((P.x1 - P.x0) / P.nx), dy((P.y1 - P.y0) / P.ny) {}
  size_t cells() const { return (size_t)nx * ny; }
  // conserved-variable plane k, cell (j, i)
  size_t at(int k, int j, int i) const { return ((size_t)k * ny + j) * nx + i; }
};

// ------------------------------------------------------------ base state, a1
// ln cosh(z) up to the additive constant -ln 2, which cancels in differences.
static double lncosh_shifted(double z) {
  double a = std::fabs(z);
  return a + std::log1p(std::exp(-2.0 * a));
}

// Sec. 2.2, Eq. rho0: rho0(y) = (rho_h+rho_l)/2 + (rho_h-rho_l)/2 tanh((y-y_int)/h_s);
// p0 integrates dp/dy = rho0 g_y from the anchor p(y_ref) = p_ref in closed form.
extern "C" void o_base_state(const OParams* P, double* rho0, double* p0) {
  const Grid G(*P);
  const double zr = (P->y_ref - P->y_int) / P->h_s;
  for (int j = 0; j < P->ny; ++j) {
    const double y = P->y0 + (j + 0.5) * G.dy;
    const double z = (y - P->y_int) / P->h_s;
    rho0[j] = 0.5 * (P->rho_h + P->rho_l) + 0.5 * (P->rho_h - P->rho_l) * std::tanh(z);
    const double I = 0.5 * (P->rho_h + P->rho_l) * (y - P->y_ref)
                   + 0.5 * (P->rho_h - P->rho_l) * P->h_s * (lncosh_shifted(z) - lncosh_shifted(zr));
    p0[j] = P->p_ref + P->g_y * I;
  }
}

// --------------------------------------------------------------- scheme pieces
// Conserved (rho, mx, my, E) -> primitive (rho, ux, uy, p); Eq. total_energy.
template <class R> inline void cons_to_prim(const R U[4], R W[4], double gm1) {
  W[0] = U[0];
  W[1] = U[1] / U[0];
  W[2] = U[2] / U[0];
  W[3] = gm1 * (U[3] - 0.5 * (U[1] * W[1] + U[2] * W[2]));
}

// Limited PLM slope of cell q0 from its neighbours (minmod / MC / none).
// Ties pick the backward difference; a sign change or a zero gives slope 0.
template <class R> inline R limited_slope(const R& qm, const R& q0, const R& qp, int lim) {
  R dm = q0 - qm, dp = qp - q0;
  if (lim == O_LIM_NONE) return 0.5 * (dm + dp);
  if (lim == O_LIM_MINMOD) {
    if (val(dm) > 0.0 && val(dp) > 0.0) { sig_add(val(dm) <= val(dp) ? 1 : 2); return val(dm) <= val(dp) ? dm : dp; }
    if (val(dm) < 0.0 && val(dp) < 0.0) { sig_add(val(dm) >= val(dp) ? 3 : 4); return val(dm) >= val(dp) ? dm : dp; }
    sig_add(5);
    return R(0.0);
  }
  R a = 2.0 * dm, c = 0.5 * (dm + dp), b = 2.0 * dp;
  if (val(dm) > 0.0 && val(dp) > 0.0) {
    R s = val(a) <= val(c) ? a : c;
    sig_add(6 + (val(a) <= val(c) ? 0 : 1) + (val(s) <= val(b) ? 0 : 2));
    return val(s) <= val(b) ? s : b;
  }
  if (val(dm) < 0.0 && val(dp) < 0.0) {
    R s = val(a) >= val(c) ? a : c;
    sig_add(10 + (val(a) >= val(c) ? 0 : 1) + (val(s) >= val(b) ? 0 : 2));
    return val(s) >= val(b) ? s : b;
  }
  sig_add(14);
  return R(0.0);
}

// Physical flux of the rotated state (rho, u_n, u_t, p, E).
template <class R> inline void phys_flux(const R& r, const R& u, const R& v, const R& p, const R& E, R F[4]) {
  R f0 = r * u;
  F[0] = f0;
  F[1] = f0 * u + p;
  F[2] = f0 * v;
  F[3] = u * (E + p);
}

// HLLC star-region flux F_K + S_K (U*_K - U_K) (Toro, Spruce & Speares).
template <class R> inline void star_flux(const R& r, const R& u, const R& v, const R& p, const R& E,
                                         const R& S, const R& Ss, const R& m, R F[4]) {
  R fac = m / (S - Ss);
  R f0 = r * u;
  R us3 = fac * (E / r + (Ss - u) * (Ss + p / m));
  F[0] = f0 + S * (fac - r);
  F[1] = (f0 * u + p) + S * (fac * Ss - f0);
  F[2] = f0 * v + S * (fac * v - r * v);
  F[3] = u * (E + p) + S * (us3 - E);
}

// HLLC Riemann flux with Davis wave-speed estimates, rotated frame
// L, Rr = (rho, u_n, u_t, p). Sec. 2.3 (Godunov-type, HLLC).
template <class R> inline void hllc(const R L[4], const R Rr[4], double gamma, double gm1, R F[4]) {
  const R &rL = L[0], &uL = L[1], &vL = L[2], &pL = L[3];
  const R &rR = Rr[0], &uR = Rr[1], &vR = Rr[2], &pR = Rr[3];
  R cL = sqrt(gamma * pL / rL);
  R cR = sqrt(gamma * pR / rR);
  R aL = uL - cL, aR = uR - cR;
  R SL = val(aL) <= val(aR) ? aL : aR;
  R bL = uL + cL, bR = uR + cR;
  R SR = val(bL) >= val(bR) ? bL : bR;
  sig_add(20 + (val(aL) <= val(aR) ? 0 : 1) + (val(bL) >= val(bR) ? 0 : 2));
  R EL = pL / gm1 + 0.5 * rL * (uL * uL + vL * vL);
  R ER = pR / gm1 + 0.5 * rR * (uR * uR + vR * vR);
  R dL = SL - uL, dR = SR - uR;
  R mL = rL * dL, mR = rR * dR;
  R Ss = ((pR - pL) + uL * mL - uR * mR) / (mL - mR);
  if (val(SL) >= 0.0) { sig_add(30); phys_flux(rL, uL, vL, pL, EL, F); return; }
  if (val(Ss) >= 0.0) { sig_add(31); star_flux(rL, uL, vL, pL, EL, SL, Ss, mL, F); return; }
  if (val(SR) >= 0.0) { sig_add(32); star_flux(rR, uR, vR, pR, ER, SR, Ss, mR, F); return; }
  sig_add(33);
  phys_flux(rR, uR, vR, pR, ER, F);
}

// HLL Riemann flux (Harten, Lax & van Leer; Toro Sec. 10.3) with the same
// Davis wave speeds, rotated frame: F_L where S_L >= 0, F_R where S_R < 0, otherwise the
// single-state average (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L).
template <class R> inline void hll(const R L[4], const R Rr[4], double gamma, double gm1, R F[4]) {
  const R &rL = L[0], &uL = L[1], &vL = L[2], &pL = L[3];
  const R &rR = Rr[0], &uR = Rr[1], &vR = Rr[2], &pR = Rr[3];
  R cL = sqrt(gamma * pL / rL);
  R cR = sqrt(gamma * pR / rR);
  R aL = uL - cL, aR = uR - cR;
  R SL = val(aL) <= val(aR) ? aL : aR;
  R bL = uL + cL, bR = uR + cR;
  R SR = val(bL) >= val(bR) ? bL : bR;
  sig_add(20 + (val(aL) <= val(aR) ? 0 : 1) + (val(bL) >= val(bR) ? 0 : 2));
  R EL = pL / gm1 + 0.5 * rL * (uL * uL + vL * vL);
  R ER = pR / gm1 + 0.5 * rR * (uR * uR + vR * vR);
  R FL[4], FR[4];
  phys_flux(rL, uL, vL, pL, EL, FL);
  phys_flux(rR, uR, vR, pR, ER, FR);
  if (val(SL) >= 0.0) { sig_add(34); for (int k = 0; k < 4; ++k) F[k] = FL[k]; return; }
  if (!(val(SR) >= 0.0)) { sig_add(36); for (int k = 0; k < 4; ++k) F[k] = FR[k]; return; }
  sig_add(35);
  const R UL[4] = {rL, rL * uL, rL * vL, EL};
  const R UR[4] = {rR, rR * uR, rR * vR, ER};
  const R D = SR - SL, SLR = SL * SR;
  for (int k = 0; k < 4; ++k) F[k] = ((SR * FL[k] - SL * FR[k]) + SLR * (UR[k] - UL[k])) / D;
}

// Riemann flux of a face [Sec. 2.3, "hybrid HLLC", which the paper does not
// define; read as]: HLLC, HLL, or the hybrid, which takes HLL where the two
// face pressures differ by more than the factor flux_theta (a strong jump,
// where HLLC's contact resolution is not wanted) and HLLC elsewhere.
template <class R> inline void riemann_flux(const R L[4], const R Rr[4], const OParams& P, R F[4]) {
  bool use_hll = P.flux == O_FLUX_HLL;
  if (P.flux == O_FLUX_HYBRID) {
    use_hll = val(L[3]) > P.flux_theta * val(Rr[3]) || val(Rr[3]) > P.flux_theta * val(L[3]);
    sig_add(40 + (use_hll ? 1 : 0));
  }
  if (use_hll) hll(L, Rr, P.gamma, P.gamma - 1.0, F);
  else hllc(L, Rr, P.gamma, P.gamma - 1.0, F);
}

// Flux through the face between cells a and b along direction dir (0 = x,
// 1 = y), from the primitive states of cells a-1, a, b, b+1.
template <class R> inline void face_flux(const R* Wm, const R* Wa, const R* Wb, const R* Wp, int dir,
                                         const OParams& P, R F[4]) {
  R WL[4], WR[4];
  for (int k = 0; k < 4; ++k) {
    R sa = limited_slope(Wm[k], Wa[k], Wb[k], P.limiter);
    R sb = limited_slope(Wa[k], Wb[k], Wp[k], P.limiter);
    WL[k] = Wa[k] + 0.5 * sa;
    WR[k] = Wb[k] - 0.5 * sb;
  }
  const int n = 1 + dir, t = 2 - dir;
  R L[4] = {WL[0], WL[n], WL[t], WL[3]};
  R Rr[4] = {WR[0], WR[n], WR[t], WR[3]};
  R f[4];
  riemann_flux(L, Rr, P, f);
  F[0] = f[0]; F[n] = f[1]; F[t] = f[2]; F[3] = f[3];
}

// Primitive variables on the grid extended by H ghost layers (cross-shaped use:
// x ghosts on interior rows, y ghosts on interior columns).
template <class R> struct Ext {
  int nx, ny, w;
  std::vector<R> W;  // [(j+H)*w + (i+H)][4]
  Ext(int nx_, int ny_) : nx(nx_), ny(ny_), w(nx_ + 2 * H), W((size_t)(nx_ + 2 * H) * (ny_ + 2 * H) * 4) {}
  R* at(int j, int i) { return &W[(((size_t)(j + H)) * w + (i + H)) * 4]; }
};

// Ghost fill in primitive variables [Sec. 2.1: periodic x; y reflecting, or
// hydrostatic with p_g = p_c + g_y rho_c (y_g - y_c)].
template <class R> static void fill_ghosts(Ext<R>& X, const OParams& P, double dy) {
  const int nx = X.nx, ny = X.ny;
  for (int j = 0; j < ny; ++j)
    for (int k = 0; k < H; ++k)
      for (int q = 0; q < 4; ++q) {
        X.at(j, -1 - k)[q] = X.at(j, nx - 1 - k)[q];
        X.at(j, nx + k)[q] = X.at(j, k)[q];
      }
  for (int i = 0; i < nx; ++i)
    for (int k = 0; k < H; ++k) {
      const double dyk = (double)(2 * k + 1) * dy;
      R* gb = X.at(-1 - k, i); const R* cb = X.at(k, i);
      R* gt = X.at(ny + k, i); const R* ct = X.at(ny - 1 - k, i);
      gb[0] = cb[0]; gb[1] = cb[1]; gb[2] = -cb[2];
      gt[0] = ct[0]; gt[1] = ct[1]; gt[2] = -ct[2];
      if (P.bc_y == O_BC_HYDROSTATIC) {
        gb[3] = cb[3] - P.g_y * cb[0] * dyk;
        gt[3] = ct[3] + P.g_y * ct[0] * dyk;
      } else {
        gb[3] = cb[3];
        gt[3] = ct[3];
      }
    }
}

template <class R> static void to_ext(const std::vector<R>& U, const Grid& G, const OParams& P, Ext<R>& X) {
  const double gm1 = P.gamma - 1.0;
#pragma omp parallel for num_threads(nthreads()) schedule(static)
  for (int j = 0; j < G.ny; ++j)
    for (int i = 0; i < G.nx; ++i) {
      R u[4] = {U[G.at(0, j, i)], U[G.at(1, j, i)], U[G.at(2, j, i)], U[G.at(3, j, i)]};
      cons_to_prim(u, X.at(j, i), gm1);
    }
  fill_ghosts(X, P, G.dy);
}

// One RK stage. out = b (stage 1) or 0.5*base + 0.5*b (stage 2) with
// b = U + (dt/dx)(F_left - F_right) + (dt/dy)(G_bottom - G_top) + dt S(U),
// S(U) = (0, 0, rho g_y, m_y g_y).                     [Eqs. mass/momentum/energy]
template <class R, class Q = double> static void stage(const OParams& P, const std::vector<R>& U, Q dt,
                                                       const std::vector<R>* base, std::vector<R>& out) {
  const Grid G(P);
  const int nx = G.nx, ny = G.ny;
  Ext<R> X(nx, ny);
  to_ext(U, G, P, X);
  std::vector<R> Fx((size_t)ny * nx * 4), Gy((size_t)(ny + 1) * nx * 4);
#pragma omp parallel for num_threads(nthreads()) schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i)  // face i: left face of cell i
      face_flux(X.at(j, i - 2), X.at(j, i - 1), X.at(j, i), X.at(j, i + 1), 0, P, &Fx[((size_t)j * nx + i) * 4]);
#pragma omp parallel for num_threads(nthreads()) schedule(static)
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i < nx; ++i)  // face j: bottom face of cell j
      face_flux(X.at(j - 2, i), X.at(j - 1, i), X.at(j, i), X.at(j + 1, i), 1, P, &Gy[((size_t)j * nx + i) * 4]);
  const Q dtdx = dt / G.dx, dtdy = dt / G.dy;
  out.resize(U.size());
#pragma omp parallel for num_threads(nthreads()) schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const R* fl = &Fx[((size_t)j * nx + i) * 4];
      const R* fr = &Fx[((size_t)j * nx + (i + 1) % nx) * 4];
      const R* gb = &Gy[((size_t)j * nx + i) * 4];
      const R* gt = &Gy[((size_t)(j + 1) * nx + i) * 4];
      for (int k = 0; k < 4; ++k) {
        R b = U[G.at(k, j, i)] + dtdx * (fl[k] - fr[k]);
        b = b + dtdy * (gb[k] - gt[k]);
        if (k == 2) b = b + dt * (U[G.at(0, j, i)] * P.g_y);
        if (k == 3) b = b + dt * (U[G.at(2, j, i)] * P.g_y);
        out[G.at(k, j, i)] = base ? 0.5 * (*base)[G.at(k, j, i)] + 0.5 * b : b;
      }
    }
}

// SSP-RK2 (Heun): U1 = U + dt L(U); U' = U/2 + (U1 + dt L(U1))/2.
template <class R, class Q = double> static void rk2_step(const OParams& P, std::vector<R>& U, Q dt) {
  std::vector<R> U1, Un;
  stage(P, U, dt, (const std::vector<R>*)nullptr, U1);
  stage(P, U1, dt, &U, Un);
  U.swap(Un);
}

// Smallest cell crossing time min(dx/(|u_x|+c), dy/(|u_y|+c)), c = sqrt(gamma p / rho).
static double cfl_wmin(const OParams& P, const std::vector<double>& U) {
  const Grid G(P);
  const double gm1 = P.gamma - 1.0;
  std::vector<double> row_min(G.ny, INFINITY);  // per-row minima, combined in row order
#pragma omp parallel for num_threads(nthreads()) schedule(static)
  for (int j = 0; j < G.ny; ++j)
    for (int i = 0; i < G.nx; ++i) {
      double u[4] = {U[G.at(0, j, i)], U[G.at(1, j, i)], U[G.at(2, j, i)], U[G.at(3, j, i)]}, W[4];
      cons_to_prim(u, W, gm1);
      const double c = std::sqrt(P.gamma * W[3] / W[0]);
      const double wx = G.dx / (std::fabs(W[1]) + c);
      const double wy = G.dy / (std::fabs(W[2]) + c);
      const double w = wx <= wy ? wx : wy;
      if (w < row_min[j]) row_min[j] = w;
    }
  double wmin = INFINITY;
  for (int j = 0; j < G.ny; ++j)
    if (row_min[j] < wmin) wmin = row_min[j];
  return wmin;
}

// Time-step control: fixed step count (nsteps > 0) or horizon T with the last
// step clipped to T - t. Returns 0 when the run is over.
static int next_dt(const OParams& P, int n, double& t, const std::vector<double>& U, double& dt) {
  if (P.nsteps > 0) {
    if (n >= P.nsteps) return 0;
    dt = P.cfl * cfl_wmin(P, U);
    t = t + dt;
    return 1;
  }
  if (t >= P.T) return 0;
  dt = P.cfl * cfl_wmin(P, U);
  const double rem = P.T - t;
  if (dt >= rem) { dt = rem; t = P.T; } else { t = t + dt; }
  return 1;
}

// Sec. 3.1: only the velocity is perturbed; rho and p keep their hydrostatic values.
template <class R> static void inject(const OParams& P, const double* rho0, const double* p0,
                                      const R* v, std::vector<R>& U) {
  const Grid G(P);
  const double gm1 = P.gamma - 1.0;
  const size_t nc = G.cells();
  U.assign(4 * nc, R(0.0));
  for (int j = 0; j < G.ny; ++j)
    for (int i = 0; i < G.nx; ++i) {
      const size_t c = (size_t)j * G.nx + i;
      R vx = P.ncomp == 2 ? v[c] : R(0.0);
      R vy = P.ncomp == 2 ? v[nc + c] : v[c];
      U[G.at(0, j, i)] = R(rho0[j]);
      U[G.at(1, j, i)] = rho0[j] * vx;
      U[G.at(2, j, i)] = rho0[j] * vy;
      U[G.at(3, j, i)] = p0[j] / gm1 + 0.5 * rho0[j] * (vx * vx + vy * vy);
    }
}

// e_k = rho |u|^2 / 2 per cell [Eq. ke]; J_KE = sum e_k dA; J_pap = sum (e_k - e_k0)^2 dA [Eq. objective].
template <class R> static R ek_cell(const R& r, const R& mx, const R& my) {
  return 0.5 * (mx * mx + my * my) / r;
}
template <class R> static void objectives(const OParams& P, const std::vector<R>& U, const double* ek0,
                                          R& J_ke, R& J_pap) {
  const Grid G(P);
  const double dA = G.dx * G.dy;
  R ske(0.0), spap(0.0);
  for (int j = 0; j < G.ny; ++j)
    for (int i = 0; i < G.nx; ++i) {
      R e = ek_cell(U[G.at(0, j, i)], U[G.at(1, j, i)], U[G.at(2, j, i)]);
      ske = ske + e;
      R a = e - (ek0 ? ek0[(size_t)j * G.nx + i] : 0.0);
      spap = spap + a * a;
    }
  J_ke = ske * dA;
  J_pap = spap * dA;
}

// ------------------------------------------------------------------ entry points
extern "C" double o_cfl_wmin(const OParams* P, const double* U) {
  const Grid G(*P);
  std::vector<double> u(U, U + 4 * G.cells());
  return cfl_wmin(*P, u);
}

// One RK stage of an arbitrary state, for unit tests: stage 1 when base is null.
extern "C" void o_stage(const OParams* P, const double* U, double dt, const double* base, double* out) {
  const Grid G(*P);
  const size_t n = 4 * G.cells();
  std::vector<double> u(U, U + n), o, b;
  if (base) { b.assign(base, base + n); stage(*P, u, dt, &b, o); }
  else stage(*P, u, dt, (const std::vector<double>*)nullptr, o);
  std::memcpy(out, o.data(), n * sizeof(double));
}

// Advance an arbitrary conserved state in place with the step control of P
// (used for Sod and conservation tests). Returns the number of steps taken.
extern "C" int o_run_state(const OParams* P, double* U, double* dt_seq, int max_steps) {
  const Grid G(*P);
  std::vector<double> u(U, U + 4 * G.cells());
  double t = 0.0, dt = 0.0;
  int n = 0;
  while (n < max_steps && next_dt(*P, n, t, u, dt)) {
    if (dt_seq) dt_seq[n] = dt;
    rk2_step(*P, u, dt);
    ++n;
  }
  std::memcpy(U, u.data(), u.size() * sizeof(double));
  return n;
}

extern "C" void o_inject(const OParams* P, const double* v, double* U) {
  const Grid G(*P);
  std::vector<double> rho0(G.ny), p0(G.ny), u;
  o_base_state(P, rho0.data(), p0.data());
  inject(*P, rho0.data(), p0.data(), v, u);
  std::memcpy(U, u.data(), u.size() * sizeof(double));
}

// Forward map F_t from the perturbation v (Sec. 3.1). When dt_replay is given
// its n_replay steps are used as the frozen step sequence; otherwise the CFL
// control of P is applied and the sequence is written to dt_seq. Outputs the
// final conserved state, e_k per cell (nullable), and J = {J_KE, J_pap}.
extern "C" int o_forward(const OParams* P, const double* v, const double* dt_replay, int n_replay,
                         double* dt_seq, int max_steps, const double* ek0,
                         double* U_out, double* ek_out, double* J) {
  const Grid G(*P);
  std::vector<double> rho0(G.ny), p0(G.ny), U;
  o_base_state(P, rho0.data(), p0.data());
  inject(*P, rho0.data(), p0.data(), v, U);
  int n = 0;
  if (dt_replay) {
    for (; n < n_replay; ++n) rk2_step(*P, U, dt_replay[n]);
  } else {
    double t = 0.0, dt = 0.0;
    while (n < max_steps && next_dt(*P, n, t, U, dt)) {
      if (dt_seq) dt_seq[n] = dt;
      rk2_step(*P, U, dt);
      ++n;
    }
  }
  if (U_out) std::memcpy(U_out, U.data(), U.size() * sizeof(double));
  if (ek_out)
    for (int j = 0; j < G.ny; ++j)
      for (int i = 0; i < G.nx; ++i)
        ek_out[(size_t)j * G.nx + i] = ek_cell(U[G.at(0, j, i)], U[G.at(1, j, i)], U[G.at(2, j, i)]);
  objectives(*P, U, ek0, J[0], J[1]);
  return n;
}

// Branch signature of the forward run from v with the frozen step sequence
// dt_replay: sig[0] = the hash of every kink decision in evaluation order,
// sig[1] = the number of decisions. Two runs with equal signatures took the
// same branch at every kink, so J is smooth between them.
extern "C" void o_forward_signature(const OParams* P, const double* v, const double* dt_replay, int n_replay,
                                    unsigned long long* sig) {
  const Grid G(*P);
  std::vector<double> rho0(G.ny), p0(G.ny), U;
  o_base_state(P, rho0.data(), p0.data());
  inject(*P, rho0.data(), p0.data(), v, U);
  g_sig = 1469598103934665603ull;
  g_sig_n = 0;
  g_sig_on = true;
  for (int n = 0; n < n_replay; ++n) rk2_step(*P, U, dt_replay[n]);
  g_sig_on = false;
  sig[0] = g_sig;
  sig[1] = (unsigned long long)g_sig_n;
}

// Directional derivative of J along dv (frozen dt sequence): forward mode.
extern "C" void o_tangent(const OParams* P, const double* v, const double* dv, const double* dt_seq,
                          int nsteps, const double* ek0, double* J, double* dJ) {
  typedef Dual<1> D;
  const Grid G(*P);
  std::vector<double> rho0(G.ny), p0(G.ny);
  o_base_state(P, rho0.data(), p0.data());
  const size_t nv = (size_t)P->ncomp * G.cells();
  std::vector<D> vd(nv);
  for (size_t c = 0; c < nv; ++c) { vd[c].v = v[c]; vd[c].d[0] = dv[c]; }
  std::vector<D> U;
  inject(*P, rho0.data(), p0.data(), vd.data(), U);
  for (int n = 0; n < nsteps; ++n) rk2_step(*P, U, dt_seq[n]);
  D jk, jp;
  objectives(*P, U, ek0, jk, jp);
  J[0] = jk.v; J[1] = jp.v;
  dJ[0] = jk.d[0]; dJ[1] = jp.d[0];
}

// Full tangent-linear state: dU(T) for the direction dv (frozen dt), used to
// assemble the tangent-linear propagator column by column on tiny grids.
extern "C" void o_tangent_state(const OParams* P, const double* v, const double* dv, const double* dt_seq,
                                int nsteps, double* U_out, double* dU_out) {
  typedef Dual<1> D;
  const Grid G(*P);
  std::vector<double> rho0(G.ny), p0(G.ny);
  o_base_state(P, rho0.data(), p0.data());
  const size_t nv = (size_t)P->ncomp * G.cells();
  std::vector<D> vd(nv);
  for (size_t c = 0; c < nv; ++c) { vd[c].v = v[c]; vd[c].d[0] = dv[c]; }
  std::vector<D> U;
  inject(*P, rho0.data(), p0.data(), vd.data(), U);
  for (int n = 0; n < nsteps; ++n) rk2_step(*P, U, dt_seq[n]);
  for (size_t q = 0; q < U.size(); ++q) { U_out[q] = U[q].v; dU_out[q] = U[q].d[0]; }
}

// ----------------------------------------------------------------- reverse mode
// Transposed stage map: out += (d b / d U)^T kap, where b is the stage value of
// stage() before the RK combination. Face flux Jacobians (4 outputs x 16
// primitive inputs) come from 16-component dual numbers; ghost cells are folded
// back onto the interior cells they copy; the primitive map is transposed per
// cell with 4-component duals.
static void stage_vjp(const OParams& P, const std::vector<double>& U, double dt,
                      const std::vector<double>& kap, std::vector<double>& out) {
  typedef Dual<16> D16;
  typedef Dual<4> D4;
  const Grid G(P);
  const int nx = G.nx, ny = G.ny;
  const double gm1 = P.gamma - 1.0;
  const double dtdx = dt / G.dx, dtdy = dt / G.dy;
  Ext<double> X(nx, ny);
  to_ext(U, G, P, X);
  Ext<double> B(nx, ny);  // cotangent of the extended primitive field
  for (auto& b : B.W) b = 0.0;

  // (dF/dW)^T mu of one face for its four cells, [cell][var]
  auto face_vjp = [&](double* w4[4], int dir, const double mu[4], double s16[16]) {
    D16 Wd[4][4];
    for (int c = 0; c < 4; ++c)
      for (int q = 0; q < 4; ++q) { Wd[c][q] = D16(w4[c][q]); Wd[c][q].d[4 * c + q] = 1.0; }
    D16 F[4];
    face_flux(Wd[0], Wd[1], Wd[2], Wd[3], dir, P, F);
    for (int c = 0; c < 4; ++c)
      for (int q = 0; q < 4; ++q) {
        double s = 0.0;
        for (int k = 0; k < 4; ++k) s += mu[k] * F[k].d[4 * c + q];
        s16[4 * c + q] = s;
      }
  };
  auto kp = [&](int k, int j, int i) { return kap[G.at(k, j, i)]; };

  // x faces: a face of row j touches only row j, so rows run in parallel
#pragma omp parallel for num_threads(nthreads()) schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {  // x face i between cells i-1 and i
      const int im = (i - 1 + nx) % nx;
      double mu[4], s16[16];
      for (int k = 0; k < 4; ++k) mu[k] = dtdx * (kp(k, j, i) - kp(k, j, im));
      double* w4[4] = {X.at(j, i - 2), X.at(j, i - 1), X.at(j, i), X.at(j, i + 1)};
      face_vjp(w4, 0, mu, s16);
      double* b4[4] = {B.at(j, i - 2), B.at(j, i - 1), B.at(j, i), B.at(j, i + 1)};
      for (int c = 0; c < 4; ++c)
        for (int q = 0; q < 4; ++q) b4[c][q] += s16[4 * c + q];
    }
  // y faces: a face touches four rows, so the faces' contributions are
  // formed in parallel and then added face by face in the serial order
  std::vector<double> Sy((size_t)(ny + 1) * nx * 16);
#pragma omp parallel for num_threads(nthreads()) schedule(static)
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i < nx; ++i) {  // y face j between cells j-1 and j
      double mu[4];
      for (int k = 0; k < 4; ++k)
        mu[k] = dtdy * ((j < ny ? kp(k, j, i) : 0.0) - (j >= 1 ? kp(k, j - 1, i) : 0.0));
      double* w4[4] = {X.at(j - 2, i), X.at(j - 1, i), X.at(j, i), X.at(j + 1, i)};
      face_vjp(w4, 1, mu, &Sy[((size_t)j * nx + i) * 16]);
    }
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const double* s16 = &Sy[((size_t)j * nx + i) * 16];
      double* b4[4] = {B.at(j - 2, i), B.at(j - 1, i), B.at(j, i), B.at(j + 1, i)};
      for (int c = 0; c < 4; ++c)
        for (int q = 0; q < 4; ++q) b4[c][q] += s16[4 * c + q];
    }
  // fold ghost cotangents onto their source cells (transpose of fill_ghosts)
  for (int j = 0; j < ny; ++j)
    for (int k = 0; k < H; ++k)
      for (int q = 0; q < 4; ++q) {
        B.at(j, nx - 1 - k)[q] += B.at(j, -1 - k)[q];
        B.at(j, k)[q] += B.at(j, nx + k)[q];
      }
  for (int i = 0; i < nx; ++i)
    for (int k = 0; k < H; ++k) {
      const double dyk = (double)(2 * k + 1) * G.dy;
      const double* gb = B.at(-1 - k, i); double* cb = B.at(k, i);
      const double* gt = B.at(ny + k, i); double* ct = B.at(ny - 1 - k, i);
      cb[0] += gb[0]; cb[1] += gb[1]; cb[2] -= gb[2]; cb[3] += gb[3];
      ct[0] += gt[0]; ct[1] += gt[1]; ct[2] -= gt[2]; ct[3] += gt[3];
      if (P.bc_y == O_BC_HYDROSTATIC) {
        cb[0] -= P.g_y * dyk * gb[3];
        ct[0] += P.g_y * dyk * gt[3];
      }
    }
  // primitive -> conserved transpose, identity part of b, gravity source
#pragma omp parallel for num_threads(nthreads()) schedule(static)
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      D4 u[4], W[4];
      for (int q = 0; q < 4; ++q) { u[q] = D4(U[G.at(q, j, i)]); u[q].d[q] = 1.0; }
      cons_to_prim(u, W, gm1);
      const double* bw = B.at(j, i);
      for (int q = 0; q < 4; ++q) {
        double s = kp(q, j, i);
        for (int m = 0; m < 4; ++m) s += bw[m] * W[m].d[q];
        out[G.at(q, j, i)] += s;
      }
      out[G.at(0, j, i)] += dt * P.g_y * kp(2, j, i);
      out[G.at(2, j, i)] += dt * P.g_y * kp(3, j, i);
    }
}

// Cotangent of the objective with respect to the final conserved state.
static void objective_cotangent(const OParams& P, const std::vector<double>& U, const double* ek0,
                                std::vector<double>& lam) {
  typedef Dual<3> D3;
  const Grid G(P);
  const double dA = G.dx * G.dy;
  lam.assign(U.size(), 0.0);
  for (int j = 0; j < G.ny; ++j)
    for (int i = 0; i < G.nx; ++i) {
      D3 r(U[G.at(0, j, i)]), mx(U[G.at(1, j, i)]), my(U[G.at(2, j, i)]);
      r.d[0] = 1.0; mx.d[1] = 1.0; my.d[2] = 1.0;
      D3 e = ek_cell(r, mx, my);
      double w = dA;
      if (P.objective == O_OBJ_PAPER) w = 2.0 * (e.v - (ek0 ? ek0[(size_t)j * G.nx + i] : 0.0)) * dA;
      for (int q = 0; q < 3; ++q) lam[G.at(q, j, i)] = w * e.d[q];
    }
}

// Reverse-mode gradient of J (P.objective) with respect to v, the dt sequence
// frozen (Sec. 3.4: the exact discrete gradient; all states stored).
// grad has the layout of v. Returns J in J[0..1] as o_forward does.
extern "C" void o_gradient(const OParams* P, const double* v, const double* dt_seq, int nsteps,
                           const double* ek0, double* J, double* grad) {
  const Grid G(*P);
  std::vector<double> rho0(G.ny), p0(G.ny);
  o_base_state(P, rho0.data(), p0.data());
  std::vector<std::vector<double>> Us(nsteps + 1);
  inject(*P, rho0.data(), p0.data(), v, Us[0]);
  for (int n = 0; n < nsteps; ++n) { Us[n + 1] = Us[n]; rk2_step(*P, Us[n + 1], dt_seq[n]); }
  objectives(*P, Us[nsteps], ek0, J[0], J[1]);
  std::vector<double> lam, lam1, lamn, U1, kap;
  objective_cotangent(*P, Us[nsteps], ek0, lam);
  for (int n = nsteps - 1; n >= 0; --n) {
    const double dt = dt_seq[n];
    stage(*P, Us[n], dt, (const std::vector<double>*)nullptr, U1);
    kap.resize(lam.size());
    for (size_t q = 0; q < lam.size(); ++q) kap[q] = 0.5 * lam[q];
    lam1.assign(lam.size(), 0.0);
    stage_vjp(*P, U1, dt, kap, lam1);
    lamn.assign(lam.size(), 0.0);
    for (size_t q = 0; q < lam.size(); ++q) lamn[q] = 0.5 * lam[q];
    stage_vjp(*P, Us[n], dt, lam1, lamn);
    lam.swap(lamn);
  }
  // transpose of inject: U1 = rho0 vx, U2 = rho0 vy, U3 += rho0 |v|^2 / 2
  const size_t nc = G.cells();
  for (int j = 0; j < G.ny; ++j)
    for (int i = 0; i < G.nx; ++i) {
      const size_t c = (size_t)j * G.nx + i;
      if (P->ncomp == 2) {
        grad[c] = rho0[j] * (lam[G.at(1, j, i)] + v[c] * lam[G.at(3, j, i)]);
        grad[nc + c] = rho0[j] * (lam[G.at(2, j, i)] + v[nc + c] * lam[G.at(3, j, i)]);
      } else {
        grad[c] = rho0[j] * (lam[G.at(2, j, i)] + v[c] * lam[G.at(3, j, i)]);
      }
    }
}

// Cotangent pull-back of one full RK2 step (for adjoint unit tests):
// lam_n = (dU^{n+1}/dU^n)^T lam.
extern "C" void o_step_vjp(const OParams* P, const double* U, double dt, const double* lam_in, double* lam_out) {
  const Grid G(*P);
  const size_t n = 4 * G.cells();
  std::vector<double> u(U, U + n), U1, lam(lam_in, lam_in + n), kap(n), lam1(n, 0.0), lamn(n);
  stage(*P, u, dt, (const std::vector<double>*)nullptr, U1);
  for (size_t q = 0; q < n; ++q) { kap[q] = 0.5 * lam[q]; lamn[q] = 0.5 * lam[q]; }
  stage_vjp(*P, U1, dt, kap, lam1);
  stage_vjp(*P, u, dt, lam1, lamn);
  std::memcpy(lam_out, lamn.data(), n * sizeof(double));
}

// ------------------------------------------- gradient through the step control
// The frozen-dt gradient above treats each dt_n as a constant. This variant
// also differentiates dt_n = cfl * min over cells and directions of the
// crossing time d / (|u_d| + c) (Sec. 2.3 CFL rule), and, in horizon mode,
// the last step dt = T - t with t = sum of the earlier steps. Readings:
//   - the derivative of the minimum is shared equally by every candidate
//     (cell, direction) whose value equals the minimum;
//   - |u| has derivative sign(u) with sign(0) = 0;
//   - the branch choices (which step is clipped) are those of the forward run.

// |a| with derivative sign(a), sign(0) = 0.
template <class R> static R abs0(const R& a) { return val(a) > 0.0 ? a : (val(a) < 0.0 ? -a : a * 0.0); }

// The candidates' mean derivative, with the (common) value kept exactly.
static double keep_value_mean(const std::vector<double>& c) { return c[0]; }
template <int N> static Dual<N> keep_value_mean(const std::vector<Dual<N>>& c) {
  Dual<N> r(c[0].v);
  for (int i = 0; i < N; ++i) {
    double s = 0.0;
    for (const auto& x : c) s += x.d[i];
    r.d[i] = s / (double)c.size();
  }
  return r;
}

// Crossing times of one cell, (d_x / (|u_x| + c), d_y / (|u_y| + c)).
template <class R> static void crossing_pair(const OParams& P, const Grid& G, const R u[4], R& wx, R& wy) {
  R W[4];
  cons_to_prim(u, W, P.gamma - 1.0);
  const R c = sqrt(P.gamma * W[3] / W[0]);
  wx = G.dx / (abs0(W[1]) + c);
  wy = G.dy / (abs0(W[2]) + c);
}

// min crossing time over the grid (its value equals cfl_wmin's).
template <class R> static R cfl_wmin_shared(const OParams& P, const std::vector<R>& U) {
  const Grid G(P);
  double wmin = INFINITY;
  std::vector<R> cand;
  for (int j = 0; j < G.ny; ++j)
    for (int i = 0; i < G.nx; ++i) {
      const R u[4] = {U[G.at(0, j, i)], U[G.at(1, j, i)], U[G.at(2, j, i)], U[G.at(3, j, i)]};
      R w[2];
      crossing_pair(P, G, u, w[0], w[1]);
      for (int d = 0; d < 2; ++d) {
        if (val(w[d]) < wmin) { wmin = val(w[d]); cand.clear(); cand.push_back(w[d]); }
        else if (val(w[d]) == wmin) cand.push_back(w[d]);
      }
    }
  return keep_value_mean(cand);
}

// lam += coef * d(min crossing time)/dU (candidates share the derivative).
static void add_wmin_gradient(const OParams& P, const std::vector<double>& U, double coef, std::vector<double>& lam) {
  typedef Dual<4> D4;
  const Grid G(P);
  const double wmin = cfl_wmin(P, U);
  std::vector<std::pair<size_t, D4>> cand;  // (cell index j*nx+i, crossing time with d/dU of that cell)
  for (int j = 0; j < G.ny; ++j)
    for (int i = 0; i < G.nx; ++i) {
      D4 u[4];
      for (int k = 0; k < 4; ++k) { u[k] = D4(U[G.at(k, j, i)]); u[k].d[k] = 1.0; }
      D4 w[2];
      crossing_pair(P, G, u, w[0], w[1]);
      for (int d = 0; d < 2; ++d)
        if (w[d].v == wmin) cand.push_back({(size_t)j * G.nx + i, w[d]});
    }
  const double share = coef / (double)cand.size();
  for (const auto& c : cand) {
    const int j = (int)(c.first / G.nx), i = (int)(c.first % G.nx);
    for (int k = 0; k < 4; ++k) lam[G.at(k, j, i)] += share * c.second.d[k];
  }
}

// Directional derivative of J along dv through the step control (forward
// mode); returns the number of steps.
extern "C" int o_tangent_dt(const OParams* P, const double* v, const double* dv, int max_steps, const double* ek0,
                            double* J, double* dJ) {
  typedef Dual<1> D;
  const Grid G(*P);
  std::vector<double> rho0(G.ny), p0(G.ny);
  o_base_state(P, rho0.data(), p0.data());
  const size_t nv = (size_t)P->ncomp * G.cells();
  std::vector<D> vd(nv);
  for (size_t c = 0; c < nv; ++c) { vd[c].v = v[c]; vd[c].d[0] = dv[c]; }
  std::vector<D> U;
  inject(*P, rho0.data(), p0.data(), vd.data(), U);
  D t(0.0);
  int n = 0;
  for (; n < max_steps; ++n) {
    if (P->nsteps > 0 ? n >= P->nsteps : t.v >= P->T) break;
    D dt = P->cfl * cfl_wmin_shared(*P, U);
    if (P->nsteps <= 0) {
      const D rem = P->T - t;
      if (dt.v >= rem.v) { dt = rem; t = D(P->T); } else { t = t + dt; }
    }
    rk2_step(*P, U, dt);
  }
  D jk, jp;
  objectives(*P, U, ek0, jk, jp);
  J[0] = jk.v; J[1] = jp.v;
  dJ[0] = jk.d[0]; dJ[1] = jp.d[0];
  return n;
}

// Reverse-mode gradient through the step control (all states stored). For
// each step n, b_n = <lam^{n+1}, dU^{n+1}/d dt_n> comes from a one-step
// forward-mode pass with dt_n as the seed; a clipped last step passes -b to
// every earlier dt; an unclipped step adds (b_n - b_last) cfl dwmin/dU^n to
// lam^n. Returns the number of steps.
extern "C" int o_gradient_dt(const OParams* P, const double* v, int max_steps, const double* ek0, double* J,
                             double* grad) {
  typedef Dual<1> D;
  const Grid G(*P);
  std::vector<double> rho0(G.ny), p0(G.ny);
  o_base_state(P, rho0.data(), p0.data());
  std::vector<std::vector<double>> Us(1);
  std::vector<double> dts;
  std::vector<char> clipped;
  inject(*P, rho0.data(), p0.data(), v, Us[0]);
  double t = 0.0, dt = 0.0;
  for (int n = 0; n < max_steps; ++n) {
    const double t_before = t;
    if (!next_dt(*P, n, t, Us[n], dt)) break;
    // the branch next_dt took: the CFL step reached the horizon and was clipped
    clipped.push_back(P->nsteps <= 0 && P->cfl * cfl_wmin(*P, Us[n]) >= P->T - t_before);
    dts.push_back(dt);
    Us.push_back(Us[n]);
    rk2_step(*P, Us[n + 1], dt);
  }
  const int N = (int)dts.size();
  objectives(*P, Us[N], ek0, J[0], J[1]);
  std::vector<double> lam, lam1, lamn, U1, kap;
  objective_cotangent(*P, Us[N], ek0, lam);
  double b_last = 0.0;
  for (int n = N - 1; n >= 0; --n) {
    // b_n = <lam^{n+1}, dU^{n+1}/d dt_n>
    std::vector<D> Ud(Us[n].begin(), Us[n].end());
    D dtd(dts[n]);
    dtd.d[0] = 1.0;
    rk2_step(*P, Ud, dtd);
    double b = 0.0;
    for (size_t q = 0; q < lam.size(); ++q) b += lam[q] * Ud[q].d[0];
    // frozen-dt pull-back of the step
    stage(*P, Us[n], dts[n], (const std::vector<double>*)nullptr, U1);
    kap.resize(lam.size());
    for (size_t q = 0; q < lam.size(); ++q) kap[q] = 0.5 * lam[q];
    lam1.assign(lam.size(), 0.0);
    stage_vjp(*P, U1, dts[n], kap, lam1);
    lamn.assign(lam.size(), 0.0);
    for (size_t q = 0; q < lam.size(); ++q) lamn[q] = 0.5 * lam[q];
    stage_vjp(*P, Us[n], dts[n], lam1, lamn);
    // dt_n = T - t_n (clipped) or cfl * wmin(U^n)
    if (clipped[n]) b_last = b;
    else add_wmin_gradient(*P, Us[n], (b - b_last) * P->cfl, lamn);
    lam.swap(lamn);
  }
  const size_t nc = G.cells();
  for (int j = 0; j < G.ny; ++j)
    for (int i = 0; i < G.nx; ++i) {
      const size_t c = (size_t)j * G.nx + i;
      if (P->ncomp == 2) {
        grad[c] = rho0[j] * (lam[G.at(1, j, i)] + v[c] * lam[G.at(3, j, i)]);
        grad[nc + c] = rho0[j] * (lam[G.at(2, j, i)] + v[nc + c] * lam[G.at(3, j, i)]);
      } else {
        grad[c] = rho0[j] * (lam[G.at(2, j, i)] + v[c] * lam[G.at(3, j, i)]);
      }
    }
  return N;
}
