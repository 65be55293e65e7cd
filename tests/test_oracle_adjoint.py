"""Pins of the oracle's derivatives: reverse sweep against forward-mode
tangents (dot-product test), tangents against central finite differences,
and the CNOP/projection machinery against the tangent-linear eigenproblem."""
import numpy as np
import pytest

import rt_inputs as I
from tests import tlm_eigen

CASES = {
    "box_minmod_ke": I.rt_box(12, 36, nsteps=30),
    "box_mc_ke_vy": I.rt_box(12, 36, nsteps=30, limiter=I.LIM_MC, ncomp=I.PERT_VY),
    "paper_hydro_pap": I.paper_unit_square(16, 0.0).replace(nsteps=30, ny=20),
    "box_none_horizon": I.rt_box(10, 30, nsteps=0, T=0.15, limiter=I.LIM_NONE),
    "box_hll_ke": I.rt_box(12, 36, nsteps=30, flux=I.FLUX_HLL),
    # theta close to 1: both branches of the switch occur
    "box_hybrid_ke": I.rt_box(12, 36, nsteps=30, flux=I.FLUX_HYBRID, flux_theta=1.0001),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_reverse_matches_tangent_on_32_directions(oracle_lib, name):
    """<grad J, d> from the reverse sweep equals J'(v) d from dual numbers to
    1e-12 relative, for 32 seeded directions (dt sequence frozen)."""
    w = CASES[name]
    o = oracle_lib
    v = o.scale_to_budget(w, I.gaussian_field(11, w.ncomp, w.ny, w.nx), 1e-3)
    ek0 = o.baseline_ek(w) if w.objective == I.OBJ_EK_ANOMALY_L2 else None
    J, g, out = o.value_and_gradient(w, v, ek0)
    D = I.directions(1000, 32, w.ncomp, w.ny, w.nx)
    worst = 0.0
    for d in D:
        Jt, dJ = o.tangent(w, v, d, out["dt"], ek0)
        assert Jt == J
        worst = max(worst, abs(np.sum(g * d) - dJ) / (abs(dJ) + 1e-300))
    assert worst <= 1e-12, worst


def test_tangent_matches_central_differences(oracle_lib):
    """Central differences of the forward map (frozen dt, limiter none so that
    kinks are rare) agree with the dual-number tangent."""
    w = I.rt_box(16, 48, nsteps=40, limiter=I.LIM_NONE)
    o = oracle_lib
    v = o.scale_to_budget(w, I.gaussian_field(2, 2, w.ny, w.nx), 1e-4)
    dt = o.forward(w, v)["dt"]
    errs = []
    for d in I.directions(1000, 8, 2, w.ny, w.nx):
        _, dJ = o.tangent(w, v, d, dt)
        h = 1e-6 * np.linalg.norm(v) / np.linalg.norm(d)
        Jp = o.forward(w, v + h * d, dt_replay=dt)["J_ke"]
        Jm = o.forward(w, v - h * d, dt_replay=dt)["J_ke"]
        errs.append(abs((Jp - Jm) / (2 * h) - dJ) / abs(dJ))
    assert np.median(errs) < 1e-6 and max(errs) < 1e-5, errs


def test_gradient_matches_central_differences_minmod(oracle_lib):
    """With the default minmod limiter kinks are frequent. Each direction is
    classified by the branch signature of its two difference runs: where
    v + h d and v - h d take the same branch at every kink, the central
    difference agrees with the reverse gradient to 2e-6; directions that
    straddle a kink are reported separately (their difference mixes two
    one-sided derivatives) and must stay a minority."""
    w = I.rt_box(12, 36, nsteps=25)
    o = oracle_lib
    v = o.scale_to_budget(w, I.gaussian_field(5, 2, w.ny, w.nx), 1e-4)
    J, g, out = o.value_and_gradient(w, v)
    smooth, kinked = [], []
    for d in I.directions(1000, 12, 2, w.ny, w.nx):
        h = 1e-7 * np.linalg.norm(v) / np.linalg.norm(d)
        Jp = o.forward(w, v + h * d, dt_replay=out["dt"])["J_ke"]
        Jm = o.forward(w, v - h * d, dt_replay=out["dt"])["J_ke"]
        gd = np.sum(g * d)
        err = abs((Jp - Jm) / (2 * h) - gd) / abs(gd)
        same = o.branch_signature(w, v + h * d, out["dt"]) == o.branch_signature(w, v - h * d, out["dt"])
        (smooth if same else kinked).append(err)
    assert len(smooth) >= 8, (smooth, kinked)
    assert max(smooth) < 2e-6, (smooth, kinked)


def test_branch_signature_counts_every_kink_and_sees_a_crossing(oracle_lib):
    """The signature records one decision per limited slope (8 per face) and
    two per HLLC evaluation (Davis speeds, flux branch), per face and stage:
    with the unlimited scheme only the two. The unperturbed box has every x
    slope exactly zero; a perturbation of 1e-10 moves them off that branch,
    which the signature sees; the same run twice gives the same signature."""
    o = oracle_lib
    w = I.rt_box(8, 24, nsteps=3)
    faces = w.nx * w.ny + (w.ny + 1) * w.nx
    dt = o.forward(w, np.zeros((2, w.ny, w.nx)))["dt"]
    zero = o.branch_signature(w, np.zeros((2, w.ny, w.nx)), dt)
    assert zero[1] == 3 * 2 * faces * 10
    lin = o.branch_signature(w.replace(limiter=I.LIM_NONE), np.zeros((2, w.ny, w.nx)), dt)
    assert lin[1] == 3 * 2 * faces * 2
    # HLL has the same two decisions per face (Davis speeds, branch); the hybrid adds its sensor
    hll = o.branch_signature(w.replace(limiter=I.LIM_NONE, flux=I.FLUX_HLL), np.zeros((2, w.ny, w.nx)), dt)
    hyb = o.branch_signature(w.replace(limiter=I.LIM_NONE, flux=I.FLUX_HYBRID), np.zeros((2, w.ny, w.nx)), dt)
    assert hll[1] == lin[1] and hll[0] != lin[0] and hyb[1] == 3 * 2 * faces * 3
    xi = I.gaussian_field(1, 2, w.ny, w.nx)
    tiny = o.branch_signature(w, 1e-10 * xi, dt)
    assert tiny[1] == zero[1] and tiny[0] != zero[0]
    assert o.branch_signature(w, 1e-10 * xi, dt) == tiny


# ---------------------------------------------------------- projection, Eq. projection
def test_projection_properties(oracle_lib):
    o = oracle_lib
    w = I.rt_box(12, 36)
    v = I.gaussian_field(1, 2, w.ny, w.nx)
    eps = 1e-4
    Pv = o.project(w, v, eps)
    assert o.constraint(w, Pv) == pytest.approx(eps, rel=1e-14)
    assert np.array_equal(o.project(w, Pv * 0.5, eps), Pv * 0.5)  # identity inside
    PPv = o.project(w, Pv, eps)
    assert np.max(np.abs(PPv - Pv)) <= 1e-15 * np.max(np.abs(Pv))
    # C is the rho0-weighted energy: doubling v multiplies it by 4
    assert o.constraint(w, 2 * v) == pytest.approx(4 * o.constraint(w, v), rel=1e-15)
    # a uniform unit vy over the box gives C = (1/2) mean(rho0) * area
    rho0, _ = o.base_state(w)
    one = np.stack([np.zeros((w.ny, w.nx)), np.ones((w.ny, w.nx))])
    area = (w.x1 - w.x0) * (w.y1 - w.y0)
    assert o.constraint(w, one) == pytest.approx(0.5 * rho0.mean() * area, rel=1e-14)


def test_random_start_budget_and_localisation(oracle_lib):
    o = oracle_lib
    w = I.rt_box(16, 48)
    v = o.random_start(w, I.gaussian_field(0, 2, w.ny, w.nx), 0.15, 1e-4)
    assert o.constraint(w, v) == pytest.approx(1e-4, rel=1e-13)
    _, y = o.cell_centres(w)
    rms = np.sqrt(np.mean(v[1] ** 2, axis=1))
    assert rms[np.abs(y) < 0.1].mean() > 5 * rms[np.abs(y) > 0.5].mean()


# ------------------------------------------------------------ spectra, Eq. fourier_coeff
def test_spectrum_single_mode_and_parseval(oracle_lib):
    o = oracle_lib
    nx, ny = 32, 8
    x = np.arange(nx)
    vy = np.zeros((ny, nx))
    vy[5] = 0.3 * np.cos(2 * np.pi * 7 * x / nx + 0.4)
    vy[2] = 0.1 * np.cos(2 * np.pi * 3 * x / nx)
    y_peak, n, E = o.spectrum(vy)
    assert y_peak == 5
    assert E[n == 7][0] == pytest.approx(1.0, abs=1e-12)
    rng = I.gaussian_field(4, 1, 1, nx)[0, 0]
    _, n, E = o.spectrum(np.tile(rng, (2, 1)))
    U = np.fft.fft(rng)
    assert np.sum(np.abs(U) ** 2) == pytest.approx(nx * np.sum(rng ** 2), rel=1e-12)
    assert np.sum(E) == pytest.approx(1.0, rel=1e-14)


def test_five_modes_keeps_a_five_mode_field(oracle_lib):
    o = oracle_lib
    w = I.rt_box(32, 12, ncomp=I.PERT_VY)
    x, y = o.cell_centres(w)
    modes = [2, 5, 6, 9, 13]
    amp = [1.0, 0.8, 0.7, 0.5, 0.3]
    f = sum(a * np.cos(2 * np.pi * m * (x - w.x0) / (w.x1 - w.x0) + 0.3 * m) for a, m in zip(amp, modes))
    v = (np.exp(-y ** 2)[:, None] * f[None, :])[None]
    v = o.scale_to_budget(w, v + 1e-3 * I.gaussian_field(1, 1, w.ny, w.nx), 1e-4)
    r, keep = o.five_modes(w, v, 1e-4)
    assert keep == modes
    assert o.constraint(w, r) == pytest.approx(1e-4, rel=1e-13)
    assert np.linalg.norm(r - v) / np.linalg.norm(v) < 5e-3


# --------------------------------------------- CNOP in the tangent-linear limit
def test_cnop_small_amplitude_matches_tangent_linear_eigenvector(oracle_lib):
    """SPG CNOP at delta = 1e-12 puts >= 99% of its W0-energy in the leading
    eigenspace of the brute-force tangent-linear problem, and 2 J / (2 C)
    matches the top eigenvalue to 1e-3. Power iteration through the reverse
    sweep (v <- W0^-1 grad J) reaches the same eigenvalue."""
    o = oracle_lib
    w = tlm_eigen.steady_case()
    lam, V, w0, dt = tlm_eigen.tlm_eigen(o, w)
    nlead = int(np.sum(lam >= lam[0] * (1 - 1e-6)))
    lead = V[:, :nlead]
    eps = 1e-12
    v0 = o.scale_to_budget(w, I.gaussian_field(21, w.ncomp, w.ny, w.nx), eps)
    res = o.spg(w, v0, eps, iters=60)
    v = res["v"].ravel()
    coef = np.linalg.lstsq(lead * np.sqrt(w0)[:, None], v * np.sqrt(w0), rcond=None)[0]
    frac = np.sum((lead @ coef) ** 2 * w0) / np.sum(v ** 2 * w0)
    assert frac >= 0.99, (frac, lam[:4])
    ratio = res["J"] / o.constraint(w, res["v"])
    assert ratio == pytest.approx(lam[0], rel=1e-3)
    # power iteration through the reverse sweep
    u = v0.ravel().copy()
    for _ in range(40):
        Jv, g = o.gradient(w, u.reshape(v0.shape), dt)
        u = g.ravel() / w0
        u *= np.sqrt(eps / o.constraint(w, u.reshape(v0.shape)))
    Jv, _ = o.gradient(w, u.reshape(v0.shape), dt)
    assert Jv / eps == pytest.approx(lam[0], rel=1e-3)


def test_objective_is_quadratic_at_small_amplitude(oracle_lib):
    """J_KE(s v) / J_KE(v) -> s^2 when the unperturbed state is steady (dt
    sequence frozen at the unperturbed one; the ratio's error is O(|v|))."""
    o = oracle_lib
    w = tlm_eigen.steady_case()
    dt = o.forward(w, np.zeros((w.ncomp, w.ny, w.nx)))["dt"]
    for amp, tol in ((1e-10, 1e-4), (1e-14, 1e-6)):
        v = o.scale_to_budget(w, I.gaussian_field(3, w.ncomp, w.ny, w.nx), amp)
        J1 = o.forward(w, v, dt_replay=dt)["J_ke"]
        J2 = o.forward(w, 2 * v, dt_replay=dt)["J_ke"]
        assert J2 / J1 == pytest.approx(4.0, rel=tol)


# ------------------------------------------ two-dimensional spectra (App. B)
def test_spectrum2d_matches_fft2_and_parseval(oracle_lib):
    o = oracle_lib
    f = I.gaussian_field(8, 1, 12, 20)[0]
    E = o.spectrum2d(f)
    F = np.fft.fft2(f)
    assert np.allclose(E, np.abs(F) ** 2 / np.sum(np.abs(F) ** 2), rtol=1e-12, atol=1e-15)
    assert np.sum(E) == pytest.approx(1.0, rel=1e-14)
    # Parseval: sum |F|^2 = N sum f^2, and a real field has E(k) = E(-k)
    assert np.sum(np.abs(F) ** 2) == pytest.approx(f.size * np.sum(f * f), rel=1e-12)
    assert np.allclose(E, np.roll(np.flip(E), 1, axis=(0, 1)), rtol=1e-12, atol=1e-15)


def test_power_reconstruct_keeps_the_dominant_pairs(oracle_lib):
    """Three mode pairs with 62 / 30 / 8 % of the energy: 90 % keeps the first
    two pairs (4 modes) exactly; 50 % keeps one pair; 100 % returns the field."""
    o = oracle_lib
    w = I.rt_box(16, 12, ncomp=I.PERT_VY)
    j = np.arange(w.nx)[None, :]
    l = np.arange(w.ny)[:, None]
    a = np.sqrt([0.62, 0.30, 0.08])
    m1 = a[0] * np.cos(2 * np.pi * (3 * j / w.nx + 1 * l / w.ny))
    m2 = a[1] * np.sin(2 * np.pi * (5 * j / w.nx - 2 * l / w.ny))
    m3 = a[2] * np.cos(2 * np.pi * (1 * j / w.nx + 4 * l / w.ny) + 0.3)
    v = (m1 + m2 + m3)[None]
    eps = 1e-4
    r, kept = o.power_reconstruct(w, v, eps, 0.9)
    assert kept == 4
    assert np.allclose(r, o.scale_to_budget(w, (m1 + m2)[None], eps), rtol=1e-10, atol=1e-14)
    r, kept = o.power_reconstruct(w, v, eps, 0.5)
    assert kept == 2
    assert np.allclose(r, o.scale_to_budget(w, m1[None], eps), rtol=1e-10, atol=1e-14)
    r, kept = o.power_reconstruct(w, v, eps, 1.0)
    assert np.allclose(r, o.scale_to_budget(w, v, eps), rtol=1e-10, atol=1e-14)


# ------------------------------- gradient through the step control (dt not frozen)
@pytest.mark.parametrize("name", sorted(CASES))
def test_dt_reverse_matches_dt_tangent(oracle_lib, name):
    """Dot-product test of the reverse sweep that also differentiates the CFL
    step control against forward-mode duals through the same control."""
    o = oracle_lib
    w = CASES[name]
    v = o.scale_to_budget(w, I.gaussian_field(3, w.ncomp, w.ny, w.nx), 1e-3)
    ek0 = o.baseline_ek(w) if w.objective == I.OBJ_EK_ANOMALY_L2 else None
    J, g, n = o.gradient_dt(w, v, ek0)
    assert J == o.objective_value(w, o.forward(w, v, ek0=ek0))
    for k in range(8):
        d = I.gaussian_field(300 + k, w.ncomp, w.ny, w.nx)
        Jt, dJ, nt = o.tangent_dt(w, v, d, ek0)
        assert nt == n and Jt == J
        assert np.sum(g * d) == pytest.approx(dJ, rel=1e-12)


def test_dt_gradient_matches_differences_of_the_cfl_controlled_map(oracle_lib):
    """Central differences of the forward map as a user runs it (CFL step
    control, horizon clipping) agree with the dt-differentiated gradient to
    1e-6, while the frozen-dt gradient misses the step-control part."""
    o = oracle_lib
    w = I.rt_box(10, 30, nsteps=0, T=0.15, limiter=I.LIM_NONE)
    v = o.scale_to_budget(w, I.gaussian_field(3, w.ncomp, w.ny, w.nx), 1e-3)
    J, g, n = o.gradient_dt(w, v)
    gf = o.gradient(w, v, o.forward(w, v)["dt"])[1]
    for k in range(4):
        d = I.gaussian_field(400 + k, w.ncomp, w.ny, w.nx)
        h = 1e-6 * np.linalg.norm(v) / np.linalg.norm(d)
        fd = (o.forward(w, v + h * d)["J_ke"] - o.forward(w, v - h * d)["J_ke"]) / (2 * h)
        assert np.sum(g * d) == pytest.approx(fd, rel=1e-6)
        assert abs(np.sum(gf * d) - fd) > 10 * abs(np.sum(g * d) - fd)


def test_dt_gradient_of_an_x_uniform_field_is_x_uniform(oracle_lib):
    """x-uniform perturbations keep every row's crossing times tied along x;
    the shared-minimum reading then gives an x-uniform gradient."""
    o = oracle_lib
    w = I.rt_box(8, 24, nsteps=12)
    col = I.gaussian_field(5, w.ncomp, w.ny, 1)
    v = o.scale_to_budget(w, np.repeat(col, w.nx, axis=2), 1e-3)
    J, g, n = o.gradient_dt(w, v)
    assert np.array_equal(g, np.repeat(g[:, :, :1], w.nx, axis=2))
    d = I.gaussian_field(6, w.ncomp, w.ny, w.nx)
    Jt, dJ, _ = o.tangent_dt(w, v, d)
    assert np.sum(g * d) == pytest.approx(dJ, rel=1e-12)
