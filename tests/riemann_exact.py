"""Exact solution of the 1D Riemann problem for the ideal-gas Euler equations.

Pin for the finite-volume oracle: Newton iteration for the star pressure from
the shock / rarefaction pressure functions, then self-similar sampling
(Toro, Riemann Solvers and Numerical Methods for Fluid Dynamics, Ch. 4). It is
pinned itself by the published star-state values in tests/golden/toro_sod.json.
"""
from __future__ import annotations

import math

import numpy as np


def _pressure_function(p, rho, pk, ck, g):
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        f = (p - pk) * math.sqrt(A / (p + B))
        df = math.sqrt(A / (B + p)) * (1.0 - 0.5 * (p - pk) / (B + p))
    else:       # rarefaction
        f = 2.0 * ck / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, g):
    """(p*, u*, rho*_L, rho*_R) for primitive states (rho, u, p)."""
    rL, uL, pL = left
    rR, uR, pR = right
    cL, cR = math.sqrt(g * pL / rL), math.sqrt(g * pR / rR)
    p = max(1e-10, 0.5 * (pL + pR))
    for _ in range(100):
        fL, dL = _pressure_function(p, rL, pL, cL, g)
        fR, dR = _pressure_function(p, rR, pR, cR, g)
        dp = (fL + fR + uR - uL) / (dL + dR)
        pn = max(1e-12, p - dp)
        if abs(pn - p) <= 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = _pressure_function(p, rL, pL, cL, g)
    fR, _ = _pressure_function(p, rR, pR, cR, g)
    u = 0.5 * (uL + uR) + 0.5 * (fR - fL)

    def rho_star(rk, pk):
        if p > pk:
            q = (g - 1.0) / (g + 1.0)
            return rk * (p / pk + q) / (q * p / pk + 1.0)
        return rk * (p / pk) ** (1.0 / g)

    return p, u, rho_star(rL, pL), rho_star(rR, pR)


def sample(left, right, g, xi):
    """Primitive (rho, u, p) at the similarity coordinates xi = (x - x0) / t."""
    rL, uL, pL = left
    rR, uR, pR = right
    ps, us, rsL, rsR = star_state(left, right, g)
    cL, cR = math.sqrt(g * pL / rL), math.sqrt(g * pR / rR)
    out = np.zeros((3, len(xi)))
    for n, s in enumerate(xi):
        if s <= us:  # left of the contact
            if ps > pL:
                SL = uL - cL * math.sqrt((g + 1) / (2 * g) * ps / pL + (g - 1) / (2 * g))
                out[:, n] = (rL, uL, pL) if s <= SL else (rsL, us, ps)
            else:
                csL = cL * (ps / pL) ** ((g - 1) / (2 * g))
                if s <= uL - cL:
                    out[:, n] = (rL, uL, pL)
                elif s >= us - csL:
                    out[:, n] = (rsL, us, ps)
                else:
                    u = 2 / (g + 1) * (cL + (g - 1) / 2 * uL + s)
                    c = 2 / (g + 1) * (cL + (g - 1) / 2 * (uL - s))
                    r = rL * (c / cL) ** (2 / (g - 1))
                    out[:, n] = (r, u, pL * (c / cL) ** (2 * g / (g - 1)))
        else:
            if ps > pR:
                SR = uR + cR * math.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g))
                out[:, n] = (rR, uR, pR) if s >= SR else (rsR, us, ps)
            else:
                csR = cR * (ps / pR) ** ((g - 1) / (2 * g))
                if s >= uR + cR:
                    out[:, n] = (rR, uR, pR)
                elif s <= us + csR:
                    out[:, n] = (rsR, us, ps)
                else:
                    u = 2 / (g + 1) * (-cR + (g - 1) / 2 * uR + s)
                    c = 2 / (g + 1) * (cR - (g - 1) / 2 * (uR - s))
                    r = rR * (c / cR) ** (2 / (g - 1))
                    out[:, n] = (r, u, pR * (c / cR) ** (2 * g / (g - 1)))
    return out
