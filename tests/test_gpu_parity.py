"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

FP64 path: the state and the dt sequence are bitwise equal to the oracle's
(same expressions, no FMA contraction); J agrees to summation order; the
gradient agrees to 1e-11 relative L2. FP32-state path: J within 1e-4
relative, gradient cosine >= 0.999 against the FP64 oracle.
"""
import numpy as np
import pytest

import rt_inputs as I

pytestmark = pytest.mark.gpu


def _rt():
    import paper_2608_04085_b300 as rt
    return rt


def _v(w, seed, amp=1e-4):
    import oracle
    return oracle.scale_to_budget(w, I.gaussian_field(seed, w.ncomp, w.ny, w.nx), amp)


FWD_CASES = {
    # 64x192 RT box, 500 CFL steps, (vx, vy) at C = 1e-4: the small workload in full
    "box64x192_500": (I.small_fixed_steps(), 0),
    # ragged tiles in x and y, MC limiter, u_y-only, hydrostatic walls
    "ragged37x45_mc_hydro": (I.rt_box(37, 45, nsteps=60, limiter=I.LIM_MC, ncomp=I.PERT_VY,
                                      bc_y=I.BC_HYDROSTATIC), 1),
    # unit square of the paper, horizon mode with the clipped last step, anomaly objective
    "paper20_horizon": (I.paper_unit_square(20, 0.05).replace(ny=27), 2),
    # minimal sizes: nx = 4, ny = 2 (a single ragged tile, mirror ghosts of 2 rows)
    "tiny4x2_none": (I.rt_box(4, 2, nsteps=7, limiter=I.LIM_NONE), 3),
    # HLL flux; the HLLC/HLL hybrid with a threshold that both branches meet
    "box32x40_hll": (I.rt_box(32, 40, nsteps=40, flux=I.FLUX_HLL), 4),
    "ragged37x45_mc_hybrid": (I.rt_box(37, 45, nsteps=40, limiter=I.LIM_MC, flux=I.FLUX_HYBRID,
                                       flux_theta=1.0001), 5),
}


VARIANTS = ["sweep", "tile", "tile8", "tile32"]


def _variant(rt, name):
    return {"sweep": rt.RT_STAGE_SWEEP, "tile": rt.RT_STAGE_TILE, "tile8": rt.RT_STAGE_TILE8,
            "tile32": rt.RT_STAGE_TILE32}[name]


@pytest.mark.parametrize("name", sorted(FWD_CASES))
@pytest.mark.parametrize("variant", VARIANTS)
def test_fp64_forward_bitwise(name, variant):
    import oracle
    w, seed = FWD_CASES[name]
    v = _v(w, seed)
    ek0 = oracle.baseline_ek(w) if w.objective == I.OBJ_EK_ANOMALY_L2 else None
    ref = oracle.forward(w, v, ek0=ek0)
    rt = _rt()
    sk = _variant(rt, variant)
    with rt.Context([w], precision=rt.RT_FP64, stage_kernel=sk) as ctx:
        assert ctx.stage_kernel()[0] == sk
        J, Jke, st = ctx.forward(v.ravel())
        dt = ctx.dt(0)
        U = ctx.state(0)
    assert st["steps"] == ref["nsteps"]
    assert np.array_equal(dt, ref["dt"]), "dt sequence differs"
    assert np.array_equal(U, ref["U"]), f"max |dU| = {np.max(np.abs(U - ref['U']))}"
    assert Jke[0] == pytest.approx(ref["J_ke"], rel=1e-13)
    assert J[0] == pytest.approx(oracle.objective_value(w, ref), rel=1e-12)


@pytest.mark.parametrize("variant", VARIANTS)
def test_fp64_batch_of_uneven_grids_matches_single_runs(variant):
    """One batched launch over uneven instances gives each instance the same
    bits as running it alone."""
    import oracle
    ws = [I.rt_box(16, 48, nsteps=0, T=0.05), I.rt_box(40, 24, nsteps=0, T=0.08, limiter=I.LIM_MC),
          I.rt_box(8, 96, nsteps=0, T=0.03, ncomp=I.PERT_VY)]
    vs = [_v(w, 10 + k) for k, w in enumerate(ws)]
    rt = _rt()
    sk = _variant(rt, variant)
    with rt.Context(ws, precision=rt.RT_FP64, stage_kernel=sk) as ctx:
        J, Jke, st = ctx.forward(np.concatenate([v.ravel() for v in vs]))
        for k, w in enumerate(ws):
            ref = oracle.forward(w, vs[k])
            assert np.array_equal(ctx.dt(k), ref["dt"])
            assert np.array_equal(ctx.state(k), ref["U"])
            assert Jke[k] == pytest.approx(ref["J_ke"], rel=1e-13)


GRAD_CASES = {
    "box24x36_minmod": I.rt_box(24, 36, nsteps=30),
    "ragged37x21_mc_hydro_vy": I.rt_box(37, 21, nsteps=25, limiter=I.LIM_MC, ncomp=I.PERT_VY,
                                        bc_y=I.BC_HYDROSTATIC),
    "paper16_pap_horizon": I.paper_unit_square(16, 0.04).replace(ny=20),
    "tiny4x2": I.rt_box(4, 2, nsteps=6, limiter=I.LIM_NONE),
    "box24x36_hll": I.rt_box(24, 36, nsteps=30, flux=I.FLUX_HLL),
    "box24x36_hybrid": I.rt_box(24, 36, nsteps=30, flux=I.FLUX_HYBRID, flux_theta=1.0001),
}


@pytest.mark.parametrize("name", sorted(GRAD_CASES))
@pytest.mark.parametrize("ckpt", ["store_all", "sqrt"])
def test_fp64_gradient_matches_oracle(name, ckpt):
    import oracle
    w = GRAD_CASES[name]
    v = _v(w, 5, 1e-3)
    ek0 = oracle.baseline_ek(w) if w.objective == I.OBJ_EK_ANOMALY_L2 else None
    Jr, gr, out = oracle.value_and_gradient(w, v, ek0)
    rt = _rt()
    mode = rt.RT_CKPT_STORE_ALL if ckpt == "store_all" else rt.RT_CKPT_SQRT
    with rt.Context([w], precision=rt.RT_FP64, ckpt=mode) as ctx:
        J, g, st = ctx.gradient(v.ravel())
        assert np.array_equal(ctx.dt(0), out["dt"])
    g = g.reshape(gr.shape)
    assert J[0] == pytest.approx(Jr, rel=1e-12)
    err = np.linalg.norm(g - gr) / np.linalg.norm(gr)
    assert err <= 1e-11, err
    if ckpt == "sqrt":
        assert st["segments"] > 1


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_checkpoint_schedules_agree_bitwise(prec):
    """Store-all, sqrt(N) and binomial checkpointing (with 0, 2 and 7 slots,
    forcing deep recomputation) give bitwise identical gradients."""
    w = I.rt_box(24, 36, nsteps=40)
    v = _v(w, 7, 1e-3).ravel()
    rt = _rt()
    p = rt.RT_FP64 if prec == "fp64" else rt.RT_FP32_STATE
    slot = 4 * w.nx * w.ny * (8 if prec == "fp64" else 4)
    runs = [(rt.RT_CKPT_STORE_ALL, 0.0), (rt.RT_CKPT_SQRT, 0.0)]
    runs += [(rt.RT_CKPT_REVOLVE, (k + 4) * slot) for k in (0, 2, 7)]
    out = []
    for mode, cap in runs:
        with rt.Context([w], precision=p, ckpt=mode, ckpt_cap_bytes=cap) as ctx:
            J, g, st = ctx.gradient(v)
            out.append((J[0], g))
            if mode == rt.RT_CKPT_REVOLVE:
                assert st["segments"] < -40  # steps were recomputed
                # exactly the optimal schedule's count (slots = cap / slot - 4)
                assert -st["segments"] == rt.revolve_plan(40, int(round(cap / slot)) - 4)[0]
    for J, g in out[1:]:
        assert J == out[0][0]
        assert np.array_equal(g, out[0][1])


def test_fp64_gradient_deterministic_and_batch_invariant():
    ws = [I.rt_box(24, 36, nsteps=20), I.rt_box(12, 20, nsteps=15, ncomp=I.PERT_VY)]
    vs = [_v(w, 3 + k, 1e-3).ravel() for k, w in enumerate(ws)]
    rt = _rt()
    with rt.Context(ws, precision=rt.RT_FP64) as ctx:
        g1 = ctx.gradient(np.concatenate(vs))[1]
        g2 = ctx.gradient(np.concatenate(vs))[1]
    assert np.array_equal(g1, g2)
    with rt.Context([ws[1]], precision=rt.RT_FP64) as ctx:
        g_single = ctx.gradient(vs[1])[1]
    assert np.array_equal(g1[vs[0].size:], g_single)


def test_fp32_state_forward_and_gradient_tolerances():
    import oracle
    w = I.rt_box(48, 96, nsteps=0, T=0.3)
    v = _v(w, 9, 1e-4)
    Jr, gr, _ = oracle.value_and_gradient(w, v)
    rt = _rt()
    with rt.Context([w], precision=rt.RT_FP32_STATE) as ctx:
        J, _, _ = ctx.forward(v.ravel())
        Jg, g, _ = ctx.gradient(v.ravel())
    assert abs(J[0] - Jr) / Jr <= 1e-4
    assert abs(Jg[0] - Jr) / Jr <= 1e-4
    g = g.reshape(gr.shape)
    cos = np.sum(g * gr) / (np.linalg.norm(g) * np.linalg.norm(gr))
    assert cos >= 0.999, cos


def test_gradient_matches_gpu_central_differences():
    """Property at any size: <g, d> = (J(v+hd) - J(v-hd)) / 2h with dt frozen
    (limiter none, so kinks are rare), evaluated with the GPU forward itself."""
    w = I.rt_box(64, 192, nsteps=120, limiter=I.LIM_NONE)
    v = _v(w, 2, 1e-4).ravel()
    rt = _rt()
    with rt.Context([w], precision=rt.RT_FP64) as ctx:
        _, g, _ = ctx.gradient(v)
        errs = []
        for d in I.directions(1000, 4, 2, w.ny, w.nx):
            d = d.ravel()
            h = 1e-6 * np.linalg.norm(v) / np.linalg.norm(d)
            ctx.forward(v)  # record the dt sequence at v
            Jp = ctx.forward(v + h * d, replay=True)[0][0]
            Jm = ctx.forward(v - h * d, replay=True)[0][0]
            errs.append(abs((Jp - Jm) / (2 * h) - g @ d) / abs(g @ d))
    assert np.median(errs) < 1e-6, errs


def test_constraint_and_projection_match_oracle():
    import oracle
    ws = [I.rt_box(24, 36), I.paper_unit_square(16)]
    vs = [I.gaussian_field(4 + k, w.ncomp, w.ny, w.nx) for k, w in enumerate(ws)]
    flat = np.concatenate([v.ravel() for v in vs])
    rt = _rt()
    with rt.Context(ws, precision=rt.RT_FP64) as ctx:
        C = ctx.constraint(flat)
        P = ctx.project(flat, [1e-4, 1e-6])
        S = ctx.project(flat * 1e-6, [1e-4, 1e-6], to_budget=True)
    off = 0
    for k, w in enumerate(ws):
        n = vs[k].size
        assert C[k] == pytest.approx(oracle.constraint(w, vs[k]), rel=1e-13)
        ref = oracle.project(w, vs[k], [1e-4, 1e-6][k]).ravel()
        assert np.max(np.abs(P[off:off + n] - ref)) <= 1e-14 * np.max(np.abs(ref))
        assert oracle.constraint(w, S[off:off + n].reshape(vs[k].shape)) == pytest.approx([1e-4, 1e-6][k], rel=1e-12)
        off += n


def test_nonfinite_state_is_reported():
    """A random perturbation far beyond the sound speed drives the pressure
    negative within five steps (the oracle shows the same); the kernels flag
    it and the call returns RT_ENONFINITE (no device fault), with the
    instance, the step and the first bad cell in the run statistics, for the
    forward and the gradient."""
    import oracle
    w = I.rt_box(16, 32, nsteps=5)
    v = 50.0 * I.gaussian_field(1, 2, w.ny, w.nx).ravel()
    rt = _rt()
    with rt.Context([w, w], precision=rt.RT_FP64) as ctx:
        vv = np.concatenate([0.0 * v, v])  # the second instance goes bad
        for call in (ctx.forward, ctx.gradient):
            with pytest.raises(rt.RtError) as e:
                call(vv)
            assert e.value.status == rt.RT_ENONFINITE
            st = e.value.stats
            assert st["bad_instance"] == 1
            assert 0 <= st["bad_step"] < 5
            assert 0 <= st["bad_cell"] < w.nx * w.ny
            assert "after step %d" % st["bad_step"] in str(e.value)
    # the step is the first whose oracle result has a non-finite or
    # non-positive density or pressure
    def valid(n):
        U = oracle.forward(w.replace(nsteps=n), v.reshape(2, w.ny, w.nx))["U"]
        p = (w.gamma - 1.0) * (U[3] - 0.5 * (U[1] ** 2 + U[2] ** 2) / U[0])
        return bool(np.all(np.isfinite(U)) and np.all(U[0] > 0) and np.all(p > 0))
    first_bad = next(n for n in range(1, 6) if not valid(n)) - 1
    assert st["bad_step"] == first_bad


def test_autotuner_picks_a_variant_and_matches_forced_ones():
    """The autotuner times the warp sweep and the tile kernel with 8-, 16- and
    32-row tiles and keeps the fastest; every variant gives the same FP32
    state to FP32 rounding (FP64 is bitwise in all, see above)."""
    w = I.rt_box(96, 160, nsteps=20)
    v = _v(w, 4).ravel()
    rt = _rt()
    out = {}
    keys = {rt.RT_STAGE_SWEEP: "sweep", rt.RT_STAGE_TILE8: "tile8", rt.RT_STAGE_TILE: "tile",
            rt.RT_STAGE_TILE32: "tile32"}
    for sk in (rt.RT_STAGE_AUTO, *keys):
        with rt.Context([w], precision=rt.RT_FP32_STATE, stage_kernel=sk) as ctx:
            var, tuned = ctx.stage_kernel()
            out[sk] = (ctx.forward(v)[0][0], ctx.state(0))
            if sk == rt.RT_STAGE_AUTO:
                assert var in keys
                assert all(t > 0 for t in tuned.values())
                assert tuned[keys[var]] == min(tuned.values())
            else:
                assert var == sk and all(t == 0 for t in tuned.values())
    # FP32 with FMA contraction: the schedules may fuse products differently,
    # so they agree to FP32 rounding (the FP64 path is bitwise in all)
    a = out[rt.RT_STAGE_TILE]
    for sk in keys:
        b = out[sk]
        assert abs(a[0] - b[0]) <= 1e-5 * abs(a[0]), sk
        assert np.max(np.abs(a[1] - b[1])) <= 1e-5 * np.max(np.abs(a[1])), sk


def test_invalid_problem_rejected():
    rt = _rt()
    with pytest.raises(rt.RtError) as e:
        rt.Context([I.rt_box(3, 8)])
    assert e.value.status == rt.RT_EINVAL


def test_mixed_flux_batch_matches_single_runs_and_bad_flux_is_rejected():
    """An HLLC, an HLL and a hybrid instance in one batch (which runs the
    generic kernels) give each instance the bits of its own oracle run, in
    FP64; the FP32 state keeps J within 1e-4 of FP64 with all three fluxes
    (the FP32 HLL average forms U_R - U_L from primitive differences). An
    unknown flux or a hybrid threshold below 1 is rejected."""
    import oracle
    rt = _rt()
    ws = [I.rt_box(24, 36, nsteps=30), I.rt_box(24, 36, nsteps=30, flux=I.FLUX_HLL),
          I.rt_box(24, 36, nsteps=30, flux=I.FLUX_HYBRID, flux_theta=1.0001)]
    vs = [_v(w, 20 + k) for k, w in enumerate(ws)]
    flat = np.concatenate([v.ravel() for v in vs])
    with rt.Context(ws, precision=rt.RT_FP64) as ctx:
        J64, _, _ = ctx.forward(flat)
        for k, w in enumerate(ws):
            ref = oracle.forward(w, vs[k])
            assert np.array_equal(ctx.state(k), ref["U"]), k
    with rt.Context(ws, precision=rt.RT_FP32_STATE) as ctx:
        J32, _, _ = ctx.forward(flat)
    rel = np.abs(J32 - J64) / np.abs(J64)
    assert np.all(rel <= 1e-4), rel
    for bad in (dict(flux=3), dict(flux=I.FLUX_HYBRID, flux_theta=0.5)):
        with pytest.raises(rt.RtError):
            rt.Context([I.rt_box(8, 8, nsteps=2, **bad)], precision=rt.RT_FP64)
