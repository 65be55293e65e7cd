"""First-order optimality (KKT) of the oracle's CNOP optimisers at finite
amplitude, where the CNOP has no closed form (Sec. 3.4). A maximiser of J on
{C <= eps} with the constraint active has C = eps and grad J = lambda grad C
with lambda > 0, grad C = rho0 v dx dy (Eq. constraint). Both the spectral
projected gradient and the projected L-BFGS must reach such a point on a
small RT box whose CNOP at eps = 1e-3 is far from the small-amplitude one;
they must agree on J and beat random perturbations of the same energy. A
gradient of the wrong sign, a projection that is not radial, or a step in
the Euclidean instead of the energy inner product (whose fixed points have
grad J parallel to v, 2% off the KKT condition here) fails these checks."""
import numpy as np
import pytest

import rt_inputs as I

EPS = 1e-3


def _case():
    # RT box with strong gravity and unlimited PLM (a smooth map, so that the
    # maximiser satisfies the classical KKT conditions)
    return I.rt_box(8, 16, nsteps=60, g_y=-1.0, limiter=I.LIM_NONE)


def _cos(a, b):
    return float(np.sum(a * b) / (np.linalg.norm(a) * np.linalg.norm(b)))


@pytest.fixture(scope="module")
def runs(oracle_lib):
    o = oracle_lib
    w = _case()
    v0 = o.scale_to_budget(w, I.gaussian_field(21, w.ncomp, w.ny, w.nx), EPS)
    return w, {"spg": o.spg(w, v0, EPS, iters=60), "lbfgs": o.lbfgs(w, v0, EPS, iters=60)}


@pytest.mark.parametrize("method", ["spg", "lbfgs"])
def test_cnop_at_finite_amplitude_is_a_kkt_point(oracle_lib, runs, method):
    o = oracle_lib
    w, res = runs
    v = res[method]["v"]
    J, g, _ = o.value_and_gradient(w, v)
    n = o.constraint_normal(w, v)
    assert o.constraint(w, v) == pytest.approx(EPS, rel=1e-12)
    assert 1.0 - _cos(g, n) <= 1e-5, 1.0 - _cos(g, n)
    assert float(np.sum(g * n)) > 0.0  # lambda > 0: the budget binds
    assert J == pytest.approx(res[method]["J"], rel=1e-14)


def test_both_optimisers_reach_the_same_maximum_above_random_starts(oracle_lib, runs):
    o = oracle_lib
    w, res = runs
    Js, Jl = res["spg"]["J"], res["lbfgs"]["J"]
    assert abs(Js - Jl) <= 1e-3 * Jl, (Js, Jl)
    rand = [o.objective_value(w, o.forward(w, o.scale_to_budget(w, I.gaussian_field(100 + k, w.ncomp, w.ny, w.nx),
                                                                    EPS)))
            for k in range(10)]
    assert min(Js, Jl) > 5.0 * max(rand), (Js, Jl, max(rand))


def test_finite_amplitude_cnop_differs_from_the_small_amplitude_one(oracle_lib, runs):
    """The regime is nonlinear: the CNOP at eps = 1e-3 is nearly orthogonal,
    in the energy inner product, to the one at eps = 1e-8 from the same start."""
    o = oracle_lib
    w, res = runs
    v0 = o.scale_to_budget(w, I.gaussian_field(21, w.ncomp, w.ny, w.nx), 1e-8)
    small = o.lbfgs(w, v0, 1e-8, iters=40)["v"].ravel()
    big = res["lbfgs"]["v"].ravel()
    wgt = o.constraint_normal(w, np.ones(big.size)).ravel()
    cos_e = float(np.sum(small * big * wgt) / np.sqrt(np.sum(small * small * wgt) * np.sum(big * big * wgt)))
    assert abs(cos_e) < 0.5, cos_e
