"""Pins of the oracle's projected L-BFGS (Sec. 3.4, Eq. projection).

- The two-loop recursion equals the dense BFGS inverse-Hessian update
  (Nocedal & Wright Eq. 6.17) applied pair by pair, and satisfies the secant
  equation H y = s for the newest pair.
- On analytic objectives the optimiser reaches the known maximiser: the
  centre of a concave quadratic with an inactive budget, and the leading
  eigenvector of a symmetric matrix on a sphere (value lambda_max r).
- On the Rayleigh-Taylor box in the small-amplitude limit the CNOP is the
  leading generalised eigenvector of the brute-force tangent-linear problem,
  the same limit that pins the spectral projected gradient.
"""
import numpy as np
import pytest

import rt_inputs as I
from tests import tlm_eigen


def _pairs(rng, n, k, skip=()):
    A = rng.standard_normal((n, n))
    A = A @ A.T + n * np.eye(n)
    out = []
    for j in range(k):
        s = rng.standard_normal(n)
        y = A @ s + 0.1 * rng.standard_normal(n)
        sy = float(s @ y)
        assert sy > 0
        out.append((s, y, 0.0 if j in skip else 1.0 / sy))
    return out


def _dense_inverse_hessian(pairs, gamma, n):
    H = gamma * np.eye(n)
    for s, y, rho in pairs:
        if rho == 0.0:
            continue
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    return H


@pytest.mark.parametrize("skip", [(), (2,), (0, 4)])
def test_two_loop_equals_dense_bfgs_update(oracle_lib, skip):
    rng = np.random.default_rng(7)
    n, k = 14, 6
    pairs = _pairs(rng, n, k, skip)
    gamma = 0.37
    H = _dense_inverse_hessian(pairs, gamma, n)
    for _ in range(3):
        g = rng.standard_normal(n)
        p = oracle_lib.lbfgs_direction(g, pairs, gamma)
        assert np.allclose(p, H @ g, rtol=1e-12, atol=1e-12 * np.linalg.norm(H @ g))
    # secant equation for the newest stored pair
    s, y, _ = [pr for pr in pairs if pr[2] > 0][-1]
    assert np.allclose(oracle_lib.lbfgs_direction(y, pairs, gamma), s, rtol=1e-11, atol=1e-11)


def test_no_pairs_gives_scaled_gradient(oracle_lib):
    g = np.arange(5.0)
    assert np.array_equal(oracle_lib.lbfgs_direction(g, [], 2.5), 2.5 * g)


def test_concave_quadratic_inactive_budget_reaches_centre(oracle_lib):
    rng = np.random.default_rng(3)
    n = 40
    B = rng.standard_normal((n, n))
    A = B @ B.T / n + 0.05 * np.eye(n)  # condition number ~ 100
    a = rng.standard_normal(n)

    def value(v):
        return -0.5 * float((v - a) @ A @ (v - a))

    def vg(v):
        return value(v), -(A @ (v - a))

    v0 = rng.standard_normal(n)
    res = oracle_lib.projected_lbfgs(value, vg, lambda v: v.copy(), v0, iters=80)
    assert np.linalg.norm(res["v"] - a) <= 1e-7 * np.linalg.norm(a)
    # with no memory (m = 0) the same loop is scaled steepest ascent, far slower
    sd = oracle_lib.projected_lbfgs(value, vg, lambda v: v.copy(), v0, iters=80, m=0)
    assert np.linalg.norm(sd["v"] - a) >= 1e-3 * np.linalg.norm(a)


def test_sphere_quadratic_reaches_leading_eigenvector(oracle_lib):
    rng = np.random.default_rng(11)
    n = 30
    B = rng.standard_normal((n, n))
    A = B @ B.T
    lam, V = np.linalg.eigh(A)
    r = 2.0

    def proj(v):
        c = float(v @ v)
        return v.copy() if c <= r else v * np.sqrt(r / c)

    def value(v):
        return float(v @ A @ v)

    def vg(v):
        return value(v), 2.0 * (A @ v)

    v0 = proj(rng.standard_normal(n) * 10)
    kw = dict(normal=lambda v: 2.0 * v, active=lambda v: float(v @ v) >= r * (1 - 1e-10))
    res = oracle_lib.projected_lbfgs(value, vg, proj, v0, iters=300, **kw)
    v = res["v"]
    cos = abs(v @ V[:, -1]) / np.linalg.norm(v)
    assert cos >= 1 - 1e-10, cos
    assert res["J"] == pytest.approx(lam[-1] * r, rel=1e-10)
    # App. A stationarity: at the maximiser g = 2 lambda v, so P(v + g) = v
    assert res["records"][-1]["chi"] <= 1e-7 * np.max(np.abs(v))
    assert res["chi0"] > 1e-2 * np.max(np.abs(v0))
    # on the sphere the pairs carry the (positive) curvature of -J o P, and the
    # quasi-Newton model converges far faster than scaled steepest ascent
    n_it = 20
    qn = oracle_lib.projected_lbfgs(value, vg, proj, v0, iters=n_it, **kw)
    sd = oracle_lib.projected_lbfgs(value, vg, proj, v0, iters=n_it, m=0, **kw)
    assert sum(rec["sy"] > 0 for rec in qn["records"]) >= n_it - 2
    gap = lambda out: lam[-1] * r - out["J"]
    assert gap(sd) > 1e-8
    assert gap(qn) <= 1e-3 * gap(sd), (gap(qn), gap(sd))


def test_monotone_memory_gives_nondecreasing_J(oracle_lib):
    o = oracle_lib
    w = I.rt_box(12, 36, nsteps=20)
    v0 = o.scale_to_budget(w, I.gaussian_field(4, w.ncomp, w.ny, w.nx), 1e-4)
    res = o.lbfgs(w, v0, 1e-4, iters=6, memory=1)
    h = res["history"]
    assert len(h) == 7
    assert all(b >= a for a, b in zip(h, h[1:])), h
    assert sum(rec["sy"] > 0 for rec in res["records"]) >= 4
    assert o.constraint(w, res["v"]) == pytest.approx(1e-4, rel=1e-12)


def test_lbfgs_small_amplitude_matches_tangent_linear_eigenvector(oracle_lib):
    """Projected L-BFGS at delta = 1e-12 puts >= 99% of its W0-energy in the
    leading eigenspace of the brute-force tangent-linear problem, and J / C
    matches the top eigenvalue to 1e-3."""
    o = oracle_lib
    w = tlm_eigen.steady_case()
    lam, V, w0, _ = tlm_eigen.tlm_eigen(o, w)
    nlead = int(np.sum(lam >= lam[0] * (1 - 1e-6)))
    lead = V[:, :nlead]
    eps = 1e-12
    v0 = o.scale_to_budget(w, I.gaussian_field(21, w.ncomp, w.ny, w.nx), eps)
    res = o.lbfgs(w, v0, eps, iters=40)
    v = res["v"].ravel()
    coef = np.linalg.lstsq(lead * np.sqrt(w0)[:, None], v * np.sqrt(w0), rcond=None)[0]
    frac = np.sum((lead @ coef) ** 2 * w0) / np.sum(v ** 2 * w0)
    assert frac >= 0.99, (frac, lam[:4])
    assert res["J"] / o.constraint(w, res["v"]) == pytest.approx(lam[0], rel=1e-3)
