"""Pins of the oracle's spectral projected gradient (Sec. 3.4, Eq. projection)
on objectives whose maximisers are known in closed form, and of its
non-monotone line search (Grippo, Lampariello & Lucidi: a trial is measured
against the worst of the last M values, so J may dip temporarily)."""
import numpy as np
import pytest


def _ball(r):
    """Radial projection onto {|v|^2 <= r} (the form of Eq. projection)."""
    def proj(v):
        c = float(v @ v)
        return v.copy() if c <= r else v * np.sqrt(r / c)
    return proj


def test_linear_objective_on_a_ball_reaches_the_boundary_point(oracle_lib):
    """max c.v over |v|^2 <= r is v* = sqrt(r) c / |c|, J* = sqrt(r) |c|."""
    rng = np.random.default_rng(1)
    c = rng.standard_normal(25)
    r = 3.0
    out = oracle_lib.projected_spg(lambda v: float(c @ v), lambda v: (float(c @ v), c.copy()), _ball(r),
                                   rng.standard_normal(25), iters=4)
    vs = np.sqrt(r) * c / np.linalg.norm(c)
    assert np.max(np.abs(out["v"] - vs)) <= 1e-14 * np.max(np.abs(vs))
    assert out["J"] == pytest.approx(np.sqrt(r) * np.linalg.norm(c), rel=1e-14)
    assert out["records"][-1]["chi"] <= 1e-14 * np.max(np.abs(vs))


def test_sphere_quadratic_reaches_the_leading_eigenvector(oracle_lib):
    """max v^T A v over |v|^2 <= r: the leading eigenvector scaled onto the
    sphere, J* = lambda_max r (eigenvalue gap 2x, so a handful of
    projected steps suffice)."""
    rng = np.random.default_rng(2)
    n = 30
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.concatenate([[10.0, 5.0], rng.uniform(1.0, 4.0, n - 2)])
    A = (Q * lam) @ Q.T
    r = 2.0
    out = oracle_lib.projected_spg(lambda v: float(v @ A @ v), lambda v: (float(v @ A @ v), 2.0 * (A @ v)),
                                   _ball(r), rng.standard_normal(n), iters=60)
    v = out["v"]
    assert abs(v @ Q[:, 0]) / np.linalg.norm(v) >= 1 - 1e-12
    assert out["J"] == pytest.approx(10.0 * r, rel=1e-12)


def test_unconstrained_concave_quadratic_and_the_non_monotone_rule(oracle_lib):
    """J = -(v - a)^T A (v - a) / 2 with no active constraint: the
    Barzilai-Borwein steps reach the centre a. With memory 10 the accepted J
    dips below the previous value at times but never below the worst of the
    last 10 values (the GLL rule); with memory 1 the sequence is monotone and,
    with backtracking cutting the BB steps, converges more slowly."""
    rng = np.random.default_rng(3)
    n = 40
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = (Q * np.geomspace(1.0, 300.0, n)) @ Q.T
    a = rng.standard_normal(n)
    J = lambda v: -0.5 * float((v - a) @ A @ (v - a))
    vg = lambda v: (J(v), -(A @ (v - a)))
    v0 = rng.standard_normal(n)
    nm = oracle_lib.projected_spg(J, vg, lambda v: v.copy(), v0, iters=300, memory=10)
    mono = oracle_lib.projected_spg(J, vg, lambda v: v.copy(), v0, iters=300, memory=1)
    err = lambda out: np.linalg.norm(out["v"] - a) / np.linalg.norm(a)
    assert err(nm) <= 1e-9 and err(mono) <= 1e-6 and err(nm) < err(mono), (err(nm), err(mono))
    h = nm["history"]
    dips = [k for k in range(1, len(h)) if h[k] < h[k - 1]]
    assert dips, "the BB steps never lowered J: the non-monotone branch was not exercised"
    assert all(h[k] >= min(h[max(0, k - 10):k]) for k in range(1, len(h)))
    hm = mono["history"]
    assert all(hm[k] >= hm[k - 1] for k in range(1, len(hm)))
