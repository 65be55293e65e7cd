"""TMA tile loads (rt_options.tile_loads = RT_LOADS_TMA, the default) against
plain loads (RT_LOADS_PLAIN): the tensor copies fetch the same values, so the
FP64 state, dt sequence and gradient are bit for bit equal, for every
stage-kernel variant, both limiter paths (minmod-specialised and generic),
uneven batches with more grid shapes than TMA groups (one instance falls
back to plain loads), y-slabs, and grids whose width is not a multiple of the
tile width. The FP64 TMA path also matches the oracle bit for bit. FP32
runs agree to rounding. A TMA wait that runs out (fault injected from the
host) ends in RT_ETIMEOUT with the device still usable."""
import numpy as np
import pytest

import rt_inputs as I

pytestmark = pytest.mark.gpu


def _rt():
    import paper_2608_04085_b300 as rt
    return rt


def _v(ws, seed, eps=1e-3):
    import oracle
    return np.concatenate([oracle.scale_to_budget(w, I.gaussian_field(seed + k, w.ncomp, w.ny, w.nx), eps).ravel()
                           for k, w in enumerate(ws)])


CASES = {
    # minmod + HLLC: the specialised kernels; 4 x 6 tiles, 2 x 3 of them by TMA
    "box128x96": [I.rt_box(128, 96, nsteps=40)],
    # MC limiter, hydrostatic walls, u_y only: the generic kernels; width 100
    # (a ragged last tile; TMA for the tiles at x0 = 32 and 64)
    "box100x90_mc_hydro": [I.rt_box(100, 90, nsteps=30, limiter=I.LIM_MC, bc_y=I.BC_HYDROSTATIC,
                                    ncomp=I.PERT_VY)],
    # five grid shapes in one batch: four TMA groups, the smallest run falls
    # back to plain loads; two equal neighbours form one group
    "uneven5": [I.rt_box(128, 96, nsteps=20), I.rt_box(128, 96, nsteps=20), I.rt_box(96, 72, nsteps=20),
                I.rt_box(160, 64, nsteps=20), I.rt_box(72, 40, nsteps=20), I.rt_box(104, 80, nsteps=20)],
}


def _variant(rt, name):
    return {"sweep": rt.RT_STAGE_SWEEP, "tile": rt.RT_STAGE_TILE, "tile8": rt.RT_STAGE_TILE8,
            "tile32": rt.RT_STAGE_TILE32}[name]


@pytest.mark.parametrize("variant", ["tile", "tile8", "tile32"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_forward_and_gradient_tma_equals_plain(name, variant):
    rt = _rt()
    ws = CASES[name]
    v = _v(ws, 7)
    out = {}
    for loads in (rt.RT_LOADS_PLAIN, rt.RT_LOADS_TMA):
        with rt.Context(ws, precision=rt.RT_FP64, stage_kernel=_variant(rt, variant), tile_loads=loads,
                        ckpt=rt.RT_CKPT_SQRT) as ctx:
            J, _, st = ctx.forward(v)
            U = [ctx.state(k) for k in range(len(ws))]
            dt = [ctx.dt(k) for k in range(len(ws))]
            Jg, g, gst = ctx.gradient(v)
            out[loads] = (J, U, dt, Jg, g, st["steps"])
    a, b = out[rt.RT_LOADS_PLAIN], out[rt.RT_LOADS_TMA]
    assert a[5] == b[5]
    for k in range(len(ws)):
        assert np.array_equal(a[2][k], b[2][k])
        assert np.array_equal(a[1][k], b[1][k]), (k, np.max(np.abs(a[1][k] - b[1][k])))
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[4], b[4]), np.max(np.abs(a[4] - b[4]))


def test_fp64_tma_matches_oracle_bitwise():
    import oracle
    rt = _rt()
    w = I.rt_box(128, 96, nsteps=25, limiter=I.LIM_MC)
    v = _v([w], 3)
    ref = oracle.forward(w, v.reshape(w.ncomp, w.ny, w.nx))
    Jr, gr = oracle.gradient(w, v.reshape(w.ncomp, w.ny, w.nx), ref["dt"])
    with rt.Context([w], precision=rt.RT_FP64, tile_loads=rt.RT_LOADS_TMA, stage_kernel=rt.RT_STAGE_TILE) as ctx:
        ctx.forward(v)
        assert np.array_equal(ctx.dt(0), ref["dt"])
        assert np.array_equal(ctx.state(0), ref["U"])
        J, g, _ = ctx.gradient(v)
    assert J[0] == pytest.approx(Jr, rel=1e-12)
    g = g.reshape(gr.shape)
    assert np.linalg.norm(g - gr) / np.linalg.norm(gr) <= 1e-11


@pytest.mark.parametrize("slabs", [2, 3])
def test_fp64_tma_with_slabs_equals_unsplit_plain(slabs):
    rt = _rt()
    w = I.rt_box(128, 160, nsteps=20)
    v = _v([w], 11)
    with rt.Context([w], precision=rt.RT_FP64, tile_loads=rt.RT_LOADS_PLAIN) as ctx:
        ctx.forward(v)
        U0, dt0 = ctx.state(0), ctx.dt(0)
        _, g0, _ = ctx.gradient(v)
    with rt.Context([w], precision=rt.RT_FP64, tile_loads=rt.RT_LOADS_TMA, y_slabs=slabs) as ctx:
        ctx.forward(v)
        assert np.array_equal(ctx.dt(0), dt0)
        assert np.array_equal(ctx.state(0), U0)
        _, g1, _ = ctx.gradient(v)
    assert np.array_equal(g1, g0)


def test_fp32_tma_agrees_with_plain():
    rt = _rt()
    ws = [I.rt_box(256, 192, nsteps=60)] * 4
    v = _v(ws, 21, 1e-4)
    out = {}
    for loads in (rt.RT_LOADS_PLAIN, rt.RT_LOADS_TMA):
        with rt.Context(ws, precision=rt.RT_FP32_STATE, tile_loads=loads, stage_kernel=rt.RT_STAGE_TILE) as ctx:
            J, _, _ = ctx.forward(v)
            _, g, _ = ctx.gradient(v)
            out[loads] = (J, g)
    Ja, ga = out[rt.RT_LOADS_PLAIN]
    Jb, gb = out[rt.RT_LOADS_TMA]
    assert np.allclose(Jb, Ja, rtol=1e-6, atol=0)
    cos = ga @ gb / (np.linalg.norm(ga) * np.linalg.norm(gb))
    assert cos >= 0.999999, cos


def test_bad_tile_loads_rejected():
    rt = _rt()
    with pytest.raises(rt.RtError) as e:
        rt.Context([I.rt_box(16, 16, nsteps=2)], precision=rt.RT_FP64, tile_loads=7)
    assert e.value.status == rt.RT_EINVAL


def test_tma_wait_that_runs_out_reports_etimeout(monkeypatch):
    """Fault injection from the host: with RT_CNOP_TMA_WAIT_FAULT=1 the tile
    kernels arm their barriers but issue no copy, so every TMA wait runs out
    after its bounded polls (nothing is in flight when the CTAs finish). The
    forward fails with RT_ETIMEOUT, and the device stays usable: a context
    without the switch then runs normally."""
    rt = _rt()
    w = I.rt_box(128, 96, nsteps=5)
    v = _v([w], 1)
    monkeypatch.setenv("RT_CNOP_TMA_WAIT_FAULT", "1")
    with rt.Context([w], precision=rt.RT_FP64, stage_kernel=rt.RT_STAGE_TILE) as ctx:
        with pytest.raises(rt.RtError) as e:
            ctx.forward(v)
        assert e.value.status == rt.RT_ETIMEOUT
    monkeypatch.delenv("RT_CNOP_TMA_WAIT_FAULT")
    with rt.Context([w], precision=rt.RT_FP64, stage_kernel=rt.RT_STAGE_TILE) as ctx:
        J, _, st = ctx.forward(v)
        assert st["steps"] == 5 and np.isfinite(J[0])
