"""Comparison diagnostics on the GPU (Sec. 4.3): KE(t) and the mixing width
h_mix(t) sampled during one forward run (rt_forward_series), against the
oracle's series, which rebuilds each sampled state by replaying the first k
time steps."""
import numpy as np
import pytest

import rt_inputs as I

pytestmark = pytest.mark.gpu


def _cases():
    return [I.rt_box(16, 48, nsteps=25), I.rt_box(24, 40, T=0.2, limiter=I.LIM_MC),
            I.paper_unit_square(20, 0.06)]


def test_series_fp64_matches_oracle():
    import oracle
    import paper_2608_04085_b300 as rt
    ws = _cases()
    vs = [oracle.scale_to_budget(w, I.gaussian_field(40 + k, w.ncomp, w.ny, w.nx), 1e-3).ravel()
          for k, w in enumerate(ws)]
    every = 4
    with rt.Context(ws, precision=rt.RT_FP64) as ctx:
        got = ctx.series(np.concatenate(vs), every)
        J, Jke, _ = ctx.forward(np.concatenate(vs))
    for k, w in enumerate(ws):
        ref = oracle.series(w, vs[k].reshape(w.ncomp, w.ny, w.nx), every)
        g = got[k]
        assert len(g["t"]) == len(ref["t"]), (len(g["t"]), ref["step"])
        assert np.allclose(g["t"], ref["t"], rtol=1e-14, atol=0)
        assert np.allclose(g["KE"], ref["KE"], rtol=1e-12, atol=0)
        assert np.allclose(g["h_mix"], ref["h_mix"], rtol=1e-12, atol=1e-15)
        assert g["KE"][-1] == pytest.approx(Jke[k], rel=1e-13)
        # singles equal the batch bitwise
        with rt.Context([w], precision=rt.RT_FP64) as c1:
            s1 = c1.series(vs[k], every)[0]
        for key in ("t", "KE", "h_mix"):
            assert np.array_equal(s1[key], g[key])


def test_series_fp32_and_limits():
    """FP32 state: KE(t) and h_mix(t) within 1e-4 of FP64; max_samples
    truncates; the unperturbed box keeps h_mix at its initial value to
    within the scheme's drift."""
    import paper_2608_04085_b300 as rt
    w = I.rt_box(32, 96, T=0.3)
    v = I.gaussian_field(3, 2, w.ny, w.nx).ravel()
    out = {}
    for prec in (rt.RT_FP64, rt.RT_FP32_STATE):
        with rt.Context([w], precision=prec) as ctx:
            v1 = ctx.project(v, 1e-4, to_budget=True)
            out[prec] = ctx.series(v1, 10)[0]
            short = ctx.series(v1, 10, max_samples=3)[0]
            assert len(short["t"]) == 3 and np.array_equal(short["KE"], out[prec]["KE"][:3])
    a, b = out[rt.RT_FP64], out[rt.RT_FP32_STATE]
    assert np.allclose(a["t"], b["t"], rtol=1e-6)
    assert np.allclose(b["KE"], a["KE"], rtol=1e-4)
    assert np.allclose(b["h_mix"], a["h_mix"], rtol=1e-4)
    with rt.Context([w], precision=rt.RT_FP64) as ctx:
        z = ctx.series(np.zeros(2 * w.nx * w.ny), 25)[0]
    assert z["KE"][0] == 0.0
    assert np.all(np.abs(z["h_mix"] - z["h_mix"][0]) <= 1e-2 * z["h_mix"][0])


def test_comparison_runs_on_the_paper_configuration():
    """Sec. 3.5 / 4.3 on a small paper configuration: a few L-BFGS iterations
    from the localised random start, then the four comparison seeds in one
    batch. The CNOP's J beats the random seed it started from; every seed
    sits on the budget; each series ends at its forward's KE."""
    import oracle
    import paper_2608_04085_b300 as rt
    from paper_2608_04085_b300.experiments import comparison_runs, SEEDS
    w = I.paper_unit_square(24, 0.1)
    eps = 1e-6
    xi = I.gaussian_field(77, w.ncomp, w.ny, w.nx).ravel()
    with rt.Context([w], precision=rt.RT_FP64) as ctx:
        v_rand = ctx.project(xi, eps, to_budget=True)
        v_loc, _, _ = ctx.cnop(xi, eps, 0, h_loc=0.1)
        v_cnop, J_cnop, res = ctx.cnop(xi, eps, 4, h_loc=0.1)
    assert res["iterations"] == 4
    out = comparison_runs(w, v_cnop, v_loc, eps, 3)
    assert set(out) == set(SEEDS)
    assert out["CNOP"]["J"] == pytest.approx(J_cnop[0], rel=1e-12)
    assert out["CNOP"]["J"] > out["Random"]["J"]
    for name in SEEDS:
        o = out[name]
        assert oracle.constraint(w, o["v"]) == pytest.approx(eps, rel=1e-12)
        assert o["KE"][-1] == pytest.approx(o["J_ke"], rel=1e-13)
        assert o["t"][-1] == pytest.approx(w.T, rel=1e-15)
        assert np.all(np.diff(o["t"]) > 0)


def test_paper_run_driver_short():
    """The paper-run driver on a cut-down budget: a batch of two seeds of the
    T2_N128 configuration, three L-BFGS iterations; every seed ends on the
    budget with J above its start and a finite KE amplification."""
    from paper_2608_04085_b300.experiments import paper_run
    out = paper_run("T2_N128", seeds=(0, 1), iters=3)
    assert out["iterations"] == 3 and out["N"] == 128
    for s in out["seeds"]:
        assert s["J_cnop"] > s["J_start"]
        assert np.isfinite(s["KE_amplification_vs_random"]) and s["KE_amplification_vs_random"] > 1.0
        assert len(s["dominant_modes"]) == 5 and all(1 <= n <= 64 for n in s["dominant_modes"])


def test_horizon_sweep_driver_short():
    """The horizon-sweep driver on short horizons and a cut-down budget: each
    horizon's CNOP ends above its random start, later horizons take more steps,
    the random start's J is the search's first J, and the five-mode seed
    has a finite positive J."""
    from paper_2608_04085_b300.experiments import horizon_sweep
    out = horizon_sweep(Ts=(0.05, 0.1), iters=2)
    assert out["iterations"] == 2 and out["grid"] == [256, 768]
    hs = out["horizons"]
    assert [h["T"] for h in hs] == [0.05, 0.1]
    assert hs[0]["steps"] < hs[1]["steps"]
    for h in hs:
        assert h["J_cnop"] > h["J_start"] > 0
        assert h["J_random"] == h["J_start"]
        assert np.isfinite(h["J_5modes"]) and h["J_5modes"] > 0


def test_precision_comparison_driver_short():
    """The FP32-vs-FP64 CNOP driver (revolve checkpointing) on a small box:
    both CNOPs rise above their common start, J of the FP64 CNOP evaluated
    in FP32 is within 1e-4, and the two CNOPs point the same way."""
    from paper_2608_04085_b300.experiments import precision_comparison
    out = precision_comparison(nx=64, ny=192, T=0.2, iters=3, ckpt_cap_gb=0.005)
    r = out["runs"]
    assert r["fp32"]["J"] > r["fp32"]["J_start"] and r["fp64"]["J"] > r["fp64"]["J_start"]
    assert abs(r["fp32"]["steps"] - r["fp64"]["steps"]) <= 1
    assert out["rel_err_J_fp32_at_fp64_cnop"] <= 1e-4
    assert out["cnop_cosine"] >= 0.999


def test_precision_comparison_fp32_search_with_fp64_checks():
    """The high-resolution mode of the driver (FP32 CNOP only, J re-evaluated
    by FP64 forwards) on a small box: J rises, and the FP32 J at the CNOP and
    at the start are within 1e-4 of the FP64 forwards."""
    from paper_2608_04085_b300.experiments import precision_comparison
    out = precision_comparison(nx=64, ny=192, T=0.2, iters=3, ckpt_cap_gb=0.005, fp64_cnop=False)
    r = out["runs"]["fp32"]
    assert r["J"] > r["J_start"] and r["revolve_recomputed_steps_per_gradient"] > 0
    assert out["rel_err_J_fp32_at_fp32_cnop"] <= 1e-4
    assert out["rel_err_J_fp32_at_start"] <= 1e-4
