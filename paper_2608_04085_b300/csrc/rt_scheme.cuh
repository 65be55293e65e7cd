// rt_scheme.cuh -- per-face arithmetic of the finite-volume scheme and of its
// adjoint, templated on the state type T (float or double).
//
// Scheme (Sec. 2.1 Eqs. mass/momentum/energy, Eq. total_energy; Sec. 2.3
// Godunov-type scheme with HLLC fluxes): PLM reconstruction of the primitive
// variables (rho, u_x, u_y, p) with a minmod / MC / unlimited slope, HLLC
// Riemann flux with Davis wave-speed estimates.
//
// Evaluation order. Every expression is written in the order in which it is
// meant to round: the FP64 translation unit is compiled with -fmad=false, so
// each product and sum rounds separately and the FP64 path reproduces an
// independent FP64 CPU implementation of the same expressions bit for bit.
// Branch conventions (all comparisons on values): minmod picks the backward
// difference on a tie and returns 0 unless both differences have the same
// strict sign; S_L = min(u_L - c_L, u_R - c_R) and S_R = max(u_L + c_L,
// u_R + c_R) pick the left argument on a tie; the HLLC branch is F_L if
// 0 <= S_L, F*_L if S_L < 0 <= S*, F*_R if S* < 0 <= S_R, F_R otherwise.
// The adjoint differentiates the branch the forward took.
#pragma once

#include <cuda_runtime.h>

namespace rt {

enum { LIM_MINMOD = 0, LIM_MC = 1, LIM_NONE = 2 };
enum { FLUX_HLLC = 0, FLUX_HLL = 1, FLUX_HYBRID = 2 };

// Riemann-flux choice of an instance (Sec. 2.3, "hybrid HLLC"): HLLC, HLL,
// or the hybrid, which takes HLL where the reconstructed face pressures
// differ by more than the factor theta and HLLC elsewhere. Kernels
// specialised for one limiter pass the constant {FLUX_HLLC, 0}, which
// removes the choice at compile time.
template <class T>
struct FluxSel {
  int kind;
  T theta;
};

template <class T>
__device__ __forceinline__ bool use_hll(const FluxSel<T>& fs, T pL, T pR) {
  if (fs.kind == FLUX_HLL) return true;
  if (fs.kind == FLUX_HYBRID) return pL > fs.theta * pR || pR > fs.theta * pL;
  return false;
}

// Conserved (rho, m_x, m_y, E) -> primitive (rho, u_x, u_y, p).
template <class T>
__device__ __forceinline__ void cons_to_prim(T r, T mx, T my, T E, T gm1, T W[4]) {
  W[0] = r;
  W[1] = mx / r;
  W[2] = my / r;
  W[3] = gm1 * (E - T(0.5) * (mx * W[1] + my * W[2]));
}

// Limited PLM slope of q0 from (qm, q0, qp).
template <class T>
__device__ __forceinline__ T limited_slope(T qm, T q0, T qp, int lim) {
  const T dm = q0 - qm, dp = qp - q0;
  if (lim == LIM_NONE) return T(0.5) * (dm + dp);
  if (lim == LIM_MINMOD) {
    // FP32: "same strict sign" as dm dp > 0 and the smaller magnitude by |dm| <= |dp|
    // (equal values; far fewer compare-and-select instructions). FP64 keeps the
    // sign tests, which also hold when dm dp underflows.
    if constexpr (sizeof(T) == 4) return (dm * dp > T(0)) ? (fabsf(dm) <= fabsf(dp) ? dm : dp) : T(0);
    if (dm > T(0) && dp > T(0)) return dm <= dp ? dm : dp;
    if (dm < T(0) && dp < T(0)) return dm >= dp ? dm : dp;
    return T(0);
  }
  const T a = T(2) * dm, c = T(0.5) * (dm + dp), b = T(2) * dp;
  if (dm > T(0) && dp > T(0)) { const T s = a <= c ? a : c; return s <= b ? s : b; }
  if (dm < T(0) && dp < T(0)) { const T s = a >= c ? a : c; return s >= b ? s : b; }
  return T(0);
}

// The same slope, also returning d slope / d (qm, q0, qp) for the branch taken.
template <class T>
__device__ __forceinline__ T limited_slope_d(T qm, T q0, T qp, int lim, T& cm, T& c0, T& cp) {
  const T dm = q0 - qm, dp = qp - q0;
  if (lim == LIM_NONE) { cm = T(-0.5); c0 = T(0); cp = T(0.5); return T(0.5) * (dm + dp); }
  if (lim == LIM_MINMOD) {
    if ((dm > T(0) && dp > T(0) && dm <= dp) || (dm < T(0) && dp < T(0) && dm >= dp)) {
      cm = T(-1); c0 = T(1); cp = T(0); return dm;
    }
    if ((dm > T(0) && dp > T(0)) || (dm < T(0) && dp < T(0))) { cm = T(0); c0 = T(-1); cp = T(1); return dp; }
    cm = c0 = cp = T(0);
    return T(0);
  }
  const T a = T(2) * dm, c = T(0.5) * (dm + dp), b = T(2) * dp;
  int pick = -1;  // 0: a, 1: c, 2: b
  if (dm > T(0) && dp > T(0)) { const bool ac = a <= c; const T s = ac ? a : c; pick = (s <= b) ? (ac ? 0 : 1) : 2; }
  else if (dm < T(0) && dp < T(0)) { const bool ac = a >= c; const T s = ac ? a : c; pick = (s >= b) ? (ac ? 0 : 1) : 2; }
  if (pick == 0) { cm = T(-2); c0 = T(2); cp = T(0); return a; }
  if (pick == 1) { cm = T(-0.5); c0 = T(0); cp = T(0.5); return c; }
  if (pick == 2) { cm = T(0); c0 = T(-2); cp = T(2); return b; }
  cm = c0 = cp = T(0);
  return T(0);
}

// HLLC flux in the frame (normal, tangential): F = (mass, normal momentum,
// tangential momentum, energy).
template <class T>
__device__ __forceinline__ void hllc(T rL, T uL, T vL, T pL, T rR, T uR, T vR, T pR,
                                     T gamma, T gm1, T F[4]) {
  const T cL = sqrt(gamma * pL / rL);
  const T cR = sqrt(gamma * pR / rR);
  const T aL = uL - cL, aR = uR - cR;
  const T SL = aL <= aR ? aL : aR;
  const T bL = uL + cL, bR = uR + cR;
  const T SR = bL >= bR ? bL : bR;
  const T dL = SL - uL, dR = SR - uR;
  const T mL = rL * dL, mR = rR * dR;
  const T Ss = ((pR - pL) + uL * mL - uR * mR) / (mL - mR);
  const bool left = (SL >= T(0)) || (Ss >= T(0));
  const bool star = left ? !(SL >= T(0)) : (SR >= T(0));
  const T r = left ? rL : rR, u = left ? uL : uR, v = left ? vL : vR, p = left ? pL : pR;
  const T S = left ? SL : SR, m = left ? mL : mR;
  // total energy of the side whose flux is taken (the other side's is not needed)
  const T E = p / gm1 + T(0.5) * r * (u * u + v * v);
  const T f0 = r * u;
  F[0] = f0;
  F[1] = f0 * u + p;
  F[2] = f0 * v;
  F[3] = u * (E + p);
  if constexpr (sizeof(T) == 4) {
    // FP32: S (U* - U) written with q = rho*/rho - 1 = (S* - u) / (S - S*),
    // U* - U = q (rho, rho S, rho v, E + p + m S*): the same values as the
    // textbook form below (which FP64 keeps, in the oracle's order), without
    // forming rho* - rho and E* - E as small differences of O(1) numbers.
    // Evaluated on every face with q = 0 off the star branches (no branch:
    // nearly every face of a subsonic flow takes a star state anyway).
    const T D = star ? S - Ss : T(1);
    const T q = star ? (Ss - u) / D : T(0);
    const T rq = r * q;
    F[0] = F[0] + S * rq;
    F[1] = F[1] + S * (rq * S);
    F[2] = F[2] + S * (rq * v);
    F[3] = F[3] + S * (q * ((E + p) + m * Ss));
    return;
  }
  if (star) {
    const T fac = m / (S - Ss);
    const T us3 = fac * (E / r + (Ss - u) * (Ss + p / m));
    F[0] = F[0] + S * (fac - r);
    F[1] = F[1] + S * (fac * Ss - f0);
    F[2] = F[2] + S * (fac * v - r * v);
    F[3] = F[3] + S * (us3 - E);
  }
}

// Reverse of hllc(): given the flux cotangent bF, return the cotangents of
// the left and right rotated primitive states (for the branch taken).
template <class T>
__device__ __forceinline__ void hllc_vjp(T rL, T uL, T vL, T pL, T rR, T uR, T vR, T pR,
                                         T gamma, T gm1, const T bF[4], T bLs[4], T bRs[4]) {
  const T cL = sqrt(gamma * pL / rL);
  const T cR = sqrt(gamma * pR / rR);
  const T aL = uL - cL, aR = uR - cR;
  const bool slL = aL <= aR;
  const T SL = slL ? aL : aR;
  const T bL = uL + cL, bR = uR + cR;
  const bool srL = bL >= bR;
  const T SR = srL ? bL : bR;
  const T dL = SL - uL, dR = SR - uR;
  const T mL = rL * dL, mR = rR * dR;
  const T den = mL - mR;
  const T Ss = ((pR - pL) + uL * mL - uR * mR) / den;
  const bool left = (SL >= T(0)) || (Ss >= T(0));
  const bool star = left ? !(SL >= T(0)) : (SR >= T(0));
  const T r = left ? rL : rR, u = left ? uL : uR, v = left ? vL : vR, p = left ? pL : pR;
  const T S = left ? SL : SR, m = left ? mL : mR;
  const T E = p / gm1 + T(0.5) * r * (u * u + v * v);
  const T f0 = r * u;

  // physical-flux part of the chosen side
  T b_f0 = bF[0] + bF[1] * u + bF[2] * v;
  T b_u = bF[1] * f0 + bF[3] * (E + p);
  T b_p = bF[1] + bF[3] * u;
  T b_v = bF[2] * f0;
  T b_E = bF[3] * u;
  T b_r = T(0), b_S = T(0), b_Ss = T(0), b_m = T(0);
  if (star) {  // + S (U* - U)
    const T D = S - Ss;
    const T fac = m / D;
    const T A = Ss - u, B = Ss + p / m;
    const T Q = E / r + A * B;
    const T us3 = fac * Q;
    b_S = bF[0] * (fac - r) + bF[1] * (fac * Ss - f0) + bF[2] * (fac * v - r * v) + bF[3] * (us3 - E);
    T b_fac = S * (bF[0] + bF[1] * Ss + bF[2] * v);
    b_r -= S * (bF[0] + bF[2] * v);
    b_Ss += S * bF[1] * fac;
    b_f0 -= S * bF[1];
    b_v += S * bF[2] * (fac - r);
    const T b_us3 = S * bF[3];
    b_E -= b_us3;
    b_fac += b_us3 * Q;
    const T b_Q = b_us3 * fac;
    b_E += b_Q / r;
    b_r -= b_Q * E / (r * r);
    const T b_A = b_Q * B, b_B = b_Q * A;
    b_Ss += b_A + b_B;
    b_u -= b_A;
    b_p += b_B / m;
    b_m -= b_B * p / (m * m);
    b_m += b_fac / D;
    const T b_D = -b_fac * fac / D;
    b_S += b_D;
    b_Ss -= b_D;
  }
  b_r += b_f0 * u;
  b_u += b_f0 * r;
  // E = p/(gamma-1) + rho (u^2 + v^2)/2 of the chosen side
  b_p += b_E / gm1;
  b_r += b_E * T(0.5) * (u * u + v * v);
  b_u += b_E * r * u;
  b_v += b_E * r * v;

  // the chosen side takes the cotangents, the other side gets zero (x - x)
  T brL = left ? b_r : T(0), buL = left ? b_u : T(0), bvL = left ? b_v : T(0);
  T bpL = left ? b_p : T(0), bSL = left ? b_S : T(0), bmL = left ? b_m : T(0);
  T brR = b_r - brL, buR = b_u - buL, bvR = b_v - bvL, bpR = b_p - bpL, bSR = b_S - bSL, bmR = b_m - bmL;
  // S* = num / den
  const T b_num = b_Ss / den;
  const T b_den = -b_Ss * Ss / den;
  bpR += b_num;
  bpL -= b_num;
  buL += b_num * mL;
  bmL += b_num * uL + b_den;
  buR -= b_num * mR;
  bmR -= b_num * uR + b_den;
  // m = rho (S - u)
  brL += bmL * dL;
  brR += bmR * dR;
  const T bdL = bmL * rL, bdR = bmR * rR;
  bSL += bdL;
  buL -= bdL;
  bSR += bdR;
  buR -= bdR;
  // Davis speeds
  const T tL = slL ? bSL : T(0), tR = bSL - tL;  // S_L = u_L - c_L or u_R - c_R
  const T sL = srL ? bSR : T(0), sR = bSR - sL;  // S_R = u_L + c_L or u_R + c_R
  buL += tL;
  buR += tR;
  buL += sL;
  buR += sR;
  const T bcL = sL - tL, bcR = sR - tR;
  // c = sqrt(gamma p / rho)
  bpL += bcL * T(0.5) * cL / pL;
  brL -= bcL * T(0.5) * cL / rL;
  bpR += bcR * T(0.5) * cR / pR;
  brR -= bcR * T(0.5) * cR / rR;
  bLs[0] = brL; bLs[1] = buL; bLs[2] = bvL; bLs[3] = bpL;
  bRs[0] = brR; bRs[1] = buR; bRs[2] = bvR; bRs[3] = bpR;
}

// FP32 reverse of hllc() differentiating the q form of the star flux that the
// FP32 forward evaluates: F = F_X + S q K for the side X whose flux is taken,
// K = (rho, rho S, rho v, E + p + m S*), q = (S* - u) / (S - S*),
// m = rho (S - u). Besides the forward's own sound speeds and S*, its only
// divisions are reciprocals formed once (of rho, c, m_L - m_R and S - S*);
// the same derivative as hllc_vjp() in exact arithmetic.
__device__ __forceinline__ void hllc_vjp_q(float rL, float uL, float vL, float pL, float rR, float uR, float vR,
                                           float pR, float gamma, float igm1, const float bF[4], float bLs[4],
                                           float bRs[4]) {
  // the quantities behind the branch choices are the forward's own
  // expressions (hllc()), so the reverse takes the branches the forward took
  const float cL = sqrt(gamma * pL / rL), cR = sqrt(gamma * pR / rR);
  const float irL = 1.0f / rL, irR = 1.0f / rR, icL = 1.0f / cL, icR = 1.0f / cR;
  const float aL = uL - cL, aR = uR - cR;
  const bool slL = aL <= aR;
  const float SL = slL ? aL : aR;
  const float eL = uL + cL, eR = uR + cR;
  const bool srL = eL >= eR;
  const float SR = srL ? eL : eR;
  const float dL = SL - uL, dR = SR - uR;
  const float mL = rL * dL, mR = rR * dR;
  const float Ss = ((pR - pL) + uL * mL - uR * mR) / (mL - mR);
  const float iden = 1.0f / (mL - mR);
  const bool left = (SL >= 0.f) || (Ss >= 0.f);
  const bool star = left ? !(SL >= 0.f) : (SR >= 0.f);
  const float r = left ? rL : rR, u = left ? uL : uR, v = left ? vL : vR, p = left ? pL : pR;
  const float S = left ? SL : SR, m = left ? mL : mR;
  const float k2 = u * u + v * v;
  const float E = p * igm1 + 0.5f * r * k2;
  const float f0 = r * u;

  // physical flux F_X = (f0, f0 u + p, f0 v, u (E + p)), f0 = rho u
  const float b_f0 = bF[0] + bF[1] * u + bF[2] * v;
  float b_u = bF[1] * f0 + bF[3] * (E + p);
  float b_p = bF[1] + bF[3] * u;
  float b_v = bF[2] * f0;
  float b_E = bF[3] * u;
  float b_r, b_S, b_Ss, b_m;
  {  // + S q K, with q = 0 and 1/D = 0 off the star branches (no branch)
    const float iD = star ? 1.0f / (S - Ss) : 0.f;
    const float q = (Ss - u) * iD;
    const float rS = r * S, rv = r * v;
    const float K3 = (E + p) + m * Ss;
    const float A = bF[0] * r + bF[1] * rS + bF[2] * rv + bF[3] * K3;  // bF . K
    const float Sq = S * q;
    const float t3 = Sq * bF[3];
    b_S = q * A + Sq * (bF[1] * r);
    b_r = Sq * (bF[0] + bF[1] * S + bF[2] * v);
    b_v += Sq * (bF[2] * r);
    b_E += t3;
    b_p += t3;
    b_m = t3 * Ss;
    b_Ss = t3 * m;
    // q = (S* - u) / (S - S*): dq/dS* = (1 + q) / D, dq/du = -1 / D, dq/dS = -q / D
    const float bqD = (S * A) * iD;
    b_Ss += bqD * (1.0f + q);
    b_u -= bqD;
    b_S -= bqD * q;
  }
  b_r += b_f0 * u;
  b_u += b_f0 * r;
  // E = p/(gamma-1) + rho (u^2 + v^2)/2 of the chosen side
  b_p += b_E * igm1;
  b_r += b_E * 0.5f * k2;
  b_u += b_E * r * u;
  b_v += b_E * r * v;

  // the chosen side takes the cotangents, the other side gets zero (x - x)
  float brL = left ? b_r : 0.f, buL = left ? b_u : 0.f, bvL = left ? b_v : 0.f;
  float bpL = left ? b_p : 0.f, bSL = left ? b_S : 0.f, bmL = left ? b_m : 0.f;
  float brR = b_r - brL, buR = b_u - buL, bvR = b_v - bvL, bpR = b_p - bpL, bSR = b_S - bSL, bmR = b_m - bmL;
  // S* = num / den, den = m_L - m_R
  const float b_num = b_Ss * iden;
  const float b_den = -b_num * Ss;
  bpR += b_num;
  bpL -= b_num;
  buL += b_num * mL;
  bmL += b_num * uL + b_den;
  buR -= b_num * mR;
  bmR -= b_num * uR + b_den;
  // m = rho (S - u)
  brL += bmL * dL;
  brR += bmR * dR;
  const float bdL = bmL * rL, bdR = bmR * rR;
  bSL += bdL;
  buL -= bdL;
  bSR += bdR;
  buR -= bdR;
  // Davis speeds
  const float tL = slL ? bSL : 0.f, tR = bSL - tL;  // S_L = u_L - c_L or u_R - c_R
  const float sL = srL ? bSR : 0.f, sR = bSR - sL;  // S_R = u_L + c_L or u_R + c_R
  buL += tL + sL;
  buR += tR + sR;
  const float bcL = sL - tL, bcR = sR - tR;
  // c = sqrt(gamma p / rho): dc/dp = gamma / (2 rho c), dc/drho = -c / (2 rho)
  const float zL = 0.5f * bcL * irL, zR = 0.5f * bcR * irR;
  bpL += zL * gamma * icL;
  brL -= zL * cL;
  bpR += zR * gamma * icR;
  brR -= zR * cR;
  bLs[0] = brL; bLs[1] = buL; bLs[2] = bvL; bLs[3] = bpL;
  bRs[0] = brR; bRs[1] = buR; bRs[2] = bvR; bRs[3] = bpR;
}

// HLL flux (Harten, Lax & van Leer) with the Davis speeds of hllc(), in
// the frame (normal, tangential): F_L where S_L >= 0, F_R where S_R < 0,
// otherwise (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L).
template <class T>
__device__ __forceinline__ void hll(T rL, T uL, T vL, T pL, T rR, T uR, T vR, T pR, T gamma, T gm1, T F[4]) {
  const T cL = sqrt(gamma * pL / rL);
  const T cR = sqrt(gamma * pR / rR);
  const T aL = uL - cL, aR = uR - cR;
  const T SL = aL <= aR ? aL : aR;
  const T eL = uL + cL, eR = uR + cR;
  const T SR = eL >= eR ? eL : eR;
  const T EL = pL / gm1 + T(0.5) * rL * (uL * uL + vL * vL);
  const T ER = pR / gm1 + T(0.5) * rR * (uR * uR + vR * vR);
  const T f0L = rL * uL, f0R = rR * uR;
  const T FL[4] = {f0L, f0L * uL + pL, f0L * vL, uL * (EL + pL)};
  const T FR[4] = {f0R, f0R * uR + pR, f0R * vR, uR * (ER + pR)};
  if (SL >= T(0)) {
#pragma unroll
    for (int k = 0; k < 4; ++k) F[k] = FL[k];
    return;
  }
  if (!(SR >= T(0))) {
#pragma unroll
    for (int k = 0; k < 4; ++k) F[k] = FR[k];
    return;
  }
  const T D = SR - SL, SLR = SL * SR;
  if constexpr (sizeof(T) == 4) {
    // FP32: U_R - U_L from differences of the primitives. p_R - p_L and
    // rho_R - rho_L of nearby face states are exact, so the diffusive term
    // rounds relative to the jump; E_R - E_L formed from the two O(1)
    // energies would round relative to the background energy p/(gamma-1).
    // The same values as the textbook form below in exact arithmetic.
    const T dU[4] = {rR - rL, rR * uR - rL * uL, rR * vR - rL * vL,
                     (pR - pL) / gm1 + T(0.5) * (rR * (uR * uR + vR * vR) - rL * (uL * uL + vL * vL))};
#pragma unroll
    for (int k = 0; k < 4; ++k) F[k] = ((SR * FL[k] - SL * FR[k]) + SLR * dU[k]) / D;
    return;
  }
  const T UL[4] = {rL, rL * uL, rL * vL, EL};
  const T UR[4] = {rR, rR * uR, rR * vR, ER};
#pragma unroll
  for (int k = 0; k < 4; ++k) F[k] = ((SR * FL[k] - SL * FR[k]) + SLR * (UR[k] - UL[k])) / D;
}

// Reverse of one side's physical flux F = (r u, r u^2 + p, r u v, u (E + p))
// and conserved state U = (r, r u, r v, E), E = p/(gamma-1) + r (u^2+v^2)/2:
// cotangents of (r, u, v, p) from those of F and U.
template <class T>
__device__ __forceinline__ void flux_state_vjp(T r, T u, T v, T p, T E, T gm1, const T bF[4], const T bU[4],
                                               T b[4]) {
  const T f0 = r * u;
  const T b_f0 = bF[0] + bF[1] * u + bF[2] * v;
  T b_u = bF[1] * f0 + bF[3] * (E + p) + b_f0 * r + bU[1] * r;
  T b_p = bF[1] + bF[3] * u;
  T b_v = bF[2] * f0 + bU[2] * r;
  const T b_E = bF[3] * u + bU[3];
  T b_r = b_f0 * u + bU[0] + bU[1] * u + bU[2] * v;
  b_p += b_E / gm1;
  b_r += b_E * T(0.5) * (u * u + v * v);
  b_u += b_E * r * u;
  b_v += b_E * r * v;
  b[0] = b_r;
  b[1] = b_u;
  b[2] = b_v;
  b[3] = b_p;
}

// Reverse of hll(): cotangents of the left and right rotated primitive
// states for the flux cotangent bF (for the branch taken). With
// D = S_R - S_L and dU = U_R - U_L: dF/dS_L = (F - F_R + S_R dU) / D,
// dF/dS_R = (F_L - F + S_L dU) / D.
template <class T>
__device__ __forceinline__ void hll_vjp(T rL, T uL, T vL, T pL, T rR, T uR, T vR, T pR, T gamma, T gm1,
                                        const T bF[4], T bLs[4], T bRs[4]) {
  const T cL = sqrt(gamma * pL / rL);
  const T cR = sqrt(gamma * pR / rR);
  const T aL = uL - cL, aR = uR - cR;
  const bool slL = aL <= aR;
  const T SL = slL ? aL : aR;
  const T eL = uL + cL, eR = uR + cR;
  const bool srL = eL >= eR;
  const T SR = srL ? eL : eR;
  const T EL = pL / gm1 + T(0.5) * rL * (uL * uL + vL * vL);
  const T ER = pR / gm1 + T(0.5) * rR * (uR * uR + vR * vR);
  const T f0L = rL * uL, f0R = rR * uR;
  const T FL[4] = {f0L, f0L * uL + pL, f0L * vL, uL * (EL + pL)};
  const T FR[4] = {f0R, f0R * uR + pR, f0R * vR, uR * (ER + pR)};
  T bFL[4], bFR[4], bUL[4], bUR[4];
  T bSL = T(0), bSR = T(0);
  const bool left = SL >= T(0), right = !left && !(SR >= T(0));
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    bFL[k] = left ? bF[k] : T(0);
    bFR[k] = right ? bF[k] : T(0);
    bUL[k] = T(0);
    bUR[k] = T(0);
  }
  if (!left && !right) {
    const T UL[4] = {rL, rL * uL, rL * vL, EL};
    const T UR[4] = {rR, rR * uR, rR * vR, ER};
    const T D = SR - SL, SLR = SL * SR;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const T dU = UR[k] - UL[k];
      const T Fk = ((SR * FL[k] - SL * FR[k]) + SLR * dU) / D;
      bFL[k] = bF[k] * SR / D;
      bFR[k] = -bF[k] * SL / D;
      bUR[k] = bF[k] * SLR / D;
      bUL[k] = -bUR[k];
      bSL += bF[k] * ((Fk - FR[k]) + SR * dU) / D;
      bSR += bF[k] * ((FL[k] - Fk) + SL * dU) / D;
    }
  }
  flux_state_vjp(rL, uL, vL, pL, EL, gm1, bFL, bUL, bLs);
  flux_state_vjp(rR, uR, vR, pR, ER, gm1, bFR, bUR, bRs);
  // Davis speeds S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R)
  const T tL = slL ? bSL : T(0), tR = bSL - tL;
  const T sL = srL ? bSR : T(0), sR = bSR - sL;
  bLs[1] += tL + sL;
  bRs[1] += tR + sR;
  const T bcL = sL - tL, bcR = sR - tR;
  // c = sqrt(gamma p / rho)
  bLs[3] += bcL * T(0.5) * cL / pL;
  bLs[0] -= bcL * T(0.5) * cL / rL;
  bRs[3] += bcR * T(0.5) * cR / pR;
  bRs[0] -= bcR * T(0.5) * cR / rR;
}

// Flux through a face along DIR (0: x, 1: y) from the reconstructed face
// states WL = W_a + s_a/2 and WR = W_b - s_b/2 (primitive, unrotated).
template <class T, int DIR>
__device__ __forceinline__ void face_flux_states(const T WL[4], const T WR[4], T gamma, T gm1, FluxSel<T> fs,
                                                 T F[4]) {
  constexpr int n = 1 + DIR, t = 2 - DIR;
  T f[4];
  if (use_hll(fs, WL[3], WR[3])) hll(WL[0], WL[n], WL[t], WL[3], WR[0], WR[n], WR[t], WR[3], gamma, gm1, f);
  else hllc(WL[0], WL[n], WL[t], WL[3], WR[0], WR[n], WR[t], WR[3], gamma, gm1, f);
  F[0] = f[0];
  F[n] = f[1];
  F[t] = f[2];
  F[3] = f[3];
}

// Flux through the face between cells a and b along DIR (0: x, 1: y), from
// the primitive states w[0..3] of cells a-1, a, b, b+1 (index [cell][var]).
template <class T, int DIR>
__device__ __forceinline__ void face_flux(const T w[4][4], int lim, T gamma, T gm1, FluxSel<T> fs, T F[4]) {
  T WL[4], WR[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const T sa = limited_slope(w[0][q], w[1][q], w[2][q], lim);
    const T sb = limited_slope(w[1][q], w[2][q], w[3][q], lim);
    WL[q] = w[1][q] + T(0.5) * sa;
    WR[q] = w[2][q] - T(0.5) * sb;
  }
  face_flux_states<T, DIR>(WL, WR, gamma, gm1, fs, F);
}

// Reverse of the HLLC part of a face: the cotangents of the reconstructed
// face states WL, WR (primitive, unrotated) for the flux cotangent mu.
template <class T, int DIR>
__device__ __forceinline__ void face_states_vjp(const T WL[4], const T WR[4], const T mu[4], T gamma, T gm1,
                                                FluxSel<T> fs, T bWL[4], T bWR[4]) {
  constexpr int n = 1 + DIR, t = 2 - DIR;
  const T bf[4] = {mu[0], mu[n], mu[t], mu[3]};
  T bl[4], br[4];
  if (use_hll(fs, WL[3], WR[3])) hll_vjp(WL[0], WL[n], WL[t], WL[3], WR[0], WR[n], WR[t], WR[3], gamma, gm1, bf, bl, br);
  else if constexpr (sizeof(T) == 4)
    hllc_vjp_q(WL[0], WL[n], WL[t], WL[3], WR[0], WR[n], WR[t], WR[3], gamma, 1.0f / gm1, bf, bl, br);
  else hllc_vjp(WL[0], WL[n], WL[t], WL[3], WR[0], WR[n], WR[t], WR[3], gamma, gm1, bf, bl, br);
  bWL[0] = bl[0]; bWL[n] = bl[1]; bWL[t] = bl[2]; bWL[3] = bl[3];
  bWR[0] = br[0]; bWR[n] = br[1]; bWR[t] = br[2]; bWR[3] = br[3];
}

// Transposed face flux: out[cell][var] = (dF/dW_cell,var)^T mu for the four
// cells a-1, a, b, b+1.
template <class T, int DIR>
__device__ __forceinline__ void face_vjp(const T w[4][4], const T mu[4], int lim, T gamma, T gm1, FluxSel<T> fs,
                                         T out[4][4]) {
  T WL[4], WR[4], bWL[4], bWR[4];
  if constexpr (sizeof(T) == 4) {
    if (lim == LIM_MINMOD) {
      // FP32 minmod in the form of limited_slope: each slope is dm (cells
      // a-1, a), dp (cells a, b) or 0, so its reverse passes the slope's
      // cotangent to the two cells of the difference it picked.
      bool nza[4], nzb[4], dma_[4], dmb_[4];  // slope nonzero; slope = dm
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const T dma = w[1][q] - w[0][q], dpa = w[2][q] - w[1][q];
        const T dmb = w[2][q] - w[1][q], dpb = w[3][q] - w[2][q];
        const bool sa = dma * dpa > T(0), sb = dmb * dpb > T(0);
        const bool ka = fabsf(dma) <= fabsf(dpa), kb = fabsf(dmb) <= fabsf(dpb);
        nza[q] = sa;
        nzb[q] = sb;
        dma_[q] = ka;
        dmb_[q] = kb;
        WL[q] = w[1][q] + T(0.5) * (sa ? (ka ? dma : dpa) : T(0));
        WR[q] = w[2][q] - T(0.5) * (sb ? (kb ? dmb : dpb) : T(0));
      }
      face_states_vjp<T, DIR>(WL, WR, mu, gamma, gm1, fs, bWL, bWR);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const T bsa = T(0.5) * bWL[q];   // W_L = W_a + s_a / 2
        const T bsb = T(-0.5) * bWR[q];  // W_R = W_b - s_b / 2
        // ta = bsa if the slope is nonzero; it goes to dm (tam) or dp (tap = ta - tam)
        const T ta = nza[q] ? bsa : T(0), tb = nzb[q] ? bsb : T(0);
        const T tam = dma_[q] ? ta : T(0), tbm = dmb_[q] ? tb : T(0);
        const T tap = ta - tam, tbp = tb - tbm;
        out[0][q] = -tam;
        out[1][q] = bWL[q] + (tam - tap) - tbm;
        out[2][q] = bWR[q] + tap + (tbm - tbp);
        out[3][q] = tbp;
      }
      return;
    }
  }
  T am[4], a0[4], ap[4], bm[4], b0[4], bp[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const T sa = limited_slope_d(w[0][q], w[1][q], w[2][q], lim, am[q], a0[q], ap[q]);
    const T sb = limited_slope_d(w[1][q], w[2][q], w[3][q], lim, bm[q], b0[q], bp[q]);
    WL[q] = w[1][q] + T(0.5) * sa;
    WR[q] = w[2][q] - T(0.5) * sb;
  }
  face_states_vjp<T, DIR>(WL, WR, mu, gamma, gm1, fs, bWL, bWR);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const T bsa = T(0.5) * bWL[q];   // W_L = W_a + s_a / 2
    const T bsb = T(-0.5) * bWR[q];  // W_R = W_b - s_b / 2
    out[0][q] = am[q] * bsa;
    out[1][q] = bWL[q] + a0[q] * bsa + bm[q] * bsb;
    out[2][q] = bWR[q] + ap[q] * bsa + b0[q] * bsb;
    out[3][q] = bp[q] * bsb;
  }
}

}  // namespace rt
