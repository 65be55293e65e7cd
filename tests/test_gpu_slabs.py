"""y-slab decomposition on the device (rt_options.y_slabs): one problem split
into 2 or 3 slabs of rows, each holding 3 halo rows per neighbouring slab,
refreshed by device-to-device copies after every kernel that writes a state
or a cotangent, with the time step, J, C and the CNOP's dot products reduced
over all slabs of the problem. Against the unsplit run of the same inputs:
state and dt sequence bit for bit, gradients bit for bit under every
checkpoint plan (every cell sums its contributions in the same order
whatever the tiling), J, C and the step-control derivative to rounding
order (their sums over cells run over other tile partitions). One GPU, one
process, no peer memory; the multi-GPU version of the same exchange is not
built."""
import numpy as np
import pytest

import rt_inputs as I

pytestmark = pytest.mark.gpu

CASES = {
    # reflecting walls, MC limiter, both velocity components, fixed steps
    "box40x60_mc": (I.rt_box(40, 60, nsteps=30, limiter=I.LIM_MC), 1e-3),
    # hydrostatic walls, u_y only, minmod, ragged tiles
    "ragged37x45_hydro_vy": (I.rt_box(37, 45, nsteps=25, bc_y=I.BC_HYDROSTATIC, ncomp=I.PERT_VY), 1e-3),
    # the paper's unit square in horizon mode with the squared e_k anomaly objective
    "paper24_horizon": (I.paper_unit_square(24, 0.06).replace(ny=30), 1e-6),
    # the HLLC/HLL hybrid (generic kernels)
    "box32x48_hybrid": (I.rt_box(32, 48, nsteps=20, flux=I.FLUX_HYBRID, flux_theta=1.0001), 1e-3),
}


def _rt():
    import paper_2608_04085_b300 as rt
    return rt


def _v(w, seed, eps):
    import oracle
    return oracle.scale_to_budget(w, I.gaussian_field(seed, w.ncomp, w.ny, w.nx), eps).ravel()


@pytest.mark.parametrize("slabs", [2, 3])
@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("variant", ["tile", "sweep", "tile8", "tile32"])
def test_fp64_forward_split_equals_unsplit(name, slabs, variant):
    rt = _rt()
    w, eps = CASES[name]
    v = _v(w, 3, eps)
    sk = {"tile": rt.RT_STAGE_TILE, "sweep": rt.RT_STAGE_SWEEP, "tile8": rt.RT_STAGE_TILE8,
          "tile32": rt.RT_STAGE_TILE32}[variant]
    out = {}
    for k in (0, slabs):
        with rt.Context([w], precision=rt.RT_FP64, stage_kernel=sk, y_slabs=k) as ctx:
            J, Jke, st = ctx.forward(v)
            out[k] = (J[0], Jke[0], ctx.dt(0), ctx.state(0), st["steps"])
    J0, K0, dt0, U0, n0 = out[0]
    J1, K1, dt1, U1, n1 = out[slabs]
    assert n1 == n0
    assert np.array_equal(dt1, dt0)
    assert np.array_equal(U1, U0), np.max(np.abs(U1 - U0))
    assert K1 == pytest.approx(K0, rel=1e-13)
    assert J1 == pytest.approx(J0, rel=1e-12)


@pytest.mark.parametrize("slabs", [2, 3])
@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_gradient_split_equals_unsplit(name, slabs):
    """Store-all, sqrt(N) and binomial checkpointing on the split problem all
    give the unsplit frozen-dt gradient bit for bit. The derivative through
    the step control adds, per step, a sum over all cells (<lam, dU/d dt>),
    whose order follows the tile partition: that gradient agrees to 1e-12."""
    rt = _rt()
    w, eps = CASES[name]
    v = _v(w, 5, eps)
    with rt.Context([w], precision=rt.RT_FP64, ckpt=rt.RT_CKPT_STORE_ALL) as ctx:
        J0, g0, _ = ctx.gradient(v)
        _, gd0, _ = ctx.gradient(v, dt_grad=True)
    slot = 4 * w.nx * (w.ny + 2 * 3 * (slabs - 1)) * 8
    for mode, cap in ((rt.RT_CKPT_STORE_ALL, 0.0), (rt.RT_CKPT_SQRT, 0.0), (rt.RT_CKPT_REVOLVE, 7 * slot)):
        with rt.Context([w], precision=rt.RT_FP64, ckpt=mode, ckpt_cap_bytes=cap, y_slabs=slabs) as ctx:
            J1, g1, _ = ctx.gradient(v)
            _, gd1, _ = ctx.gradient(v, dt_grad=True)
        assert J1[0] == pytest.approx(J0[0], rel=1e-12)
        assert np.array_equal(g1, g0), (mode, np.max(np.abs(g1 - g0)))
        err = np.linalg.norm(gd1 - gd0) / np.linalg.norm(gd0)
        assert err <= 1e-12, (mode, err)


def test_uneven_batch_split_and_fp32():
    """Two problems of different grids, each split into 3 slabs, in one batch:
    each equals its own unsplit run (FP64 bitwise); in FP32 the split and
    unsplit runs agree to FP32 rounding."""
    rt = _rt()
    ws = [I.rt_box(24, 36, nsteps=15), I.rt_box(40, 27, nsteps=12, ncomp=I.PERT_VY, limiter=I.LIM_MC)]
    vs = [_v(w, 9 + k, 1e-3) for k, w in enumerate(ws)]
    flat = np.concatenate(vs)
    with rt.Context(ws, precision=rt.RT_FP64, y_slabs=3) as ctx:
        J, _, _ = ctx.forward(flat)
        Us = [ctx.state(k) for k in range(2)]
        _, g, _ = ctx.gradient(flat)
    off = 0
    for k, w in enumerate(ws):
        with rt.Context([w], precision=rt.RT_FP64) as c1:
            Js, _, _ = c1.forward(vs[k])
            assert np.array_equal(Us[k], c1.state(0))
            _, gs, _ = c1.gradient(vs[k])
        assert J[k] == pytest.approx(Js[0], rel=1e-12)
        assert np.array_equal(g[off:off + vs[k].size], gs)
        off += vs[k].size
    out = {}
    for sl in (0, 3):
        with rt.Context(ws, precision=rt.RT_FP32_STATE, y_slabs=sl) as ctx:
            J32, _, _ = ctx.forward(flat)
            _, g32, _ = ctx.gradient(flat)
            out[sl] = (J32, g32, ctx.state(0))
    assert np.allclose(out[3][0], out[0][0], rtol=1e-6, atol=0)
    cos = out[3][1] @ out[0][1] / (np.linalg.norm(out[3][1]) * np.linalg.norm(out[0][1]))
    assert cos >= 0.999999, cos


def test_cnop_and_projection_reduce_over_slabs():
    """C, the projection and the spectral projected gradient sum over all slabs
    of the problem: the split CNOP follows the unsplit one to rounding."""
    rt = _rt()
    w = I.rt_box(24, 48, nsteps=12)
    eps = 1e-4
    xi = I.gaussian_field(4, 2, w.ny, w.nx).ravel()
    out = {}
    for k in (0, 3):
        with rt.Context([w], precision=rt.RT_FP64, y_slabs=k) as ctx:
            C = ctx.constraint(xi)
            p = ctx.project(xi, eps, to_budget=True)
            v, J, res = ctx.cnop(xi, eps, 4, method=rt.RT_CNOP_SPG, h_loc=0.2)
            assert res["status"] == rt.RT_OK
            out[k] = (C[0], p, v, J[0], res["iterations"])
    assert out[3][0] == pytest.approx(out[0][0], rel=1e-13)
    assert np.allclose(out[3][1], out[0][1], rtol=1e-13, atol=0)
    assert out[3][4] == out[0][4]
    assert out[3][3] == pytest.approx(out[0][3], rel=1e-10)
    err = np.linalg.norm(out[3][2] - out[0][2]) / np.linalg.norm(out[0][2])
    assert err <= 1e-9, err


def test_split_rejections():
    """Slabs need at least 3 rows each; the diagnostics time series, which
    reads whole rows of one instance, is not available on a split context."""
    rt = _rt()
    with pytest.raises(rt.RtError) as e:
        rt.Context([I.rt_box(8, 8, nsteps=2)], precision=rt.RT_FP64, y_slabs=3)
    assert e.value.status == rt.RT_EINVAL
    w = I.rt_box(16, 24, nsteps=4)
    with rt.Context([w], precision=rt.RT_FP64, y_slabs=2) as ctx:
        with pytest.raises(rt.RtError):
            ctx.series(_v(w, 1, 1e-3), 2)
    # unsplit problems keep the usual minimum of 2 rows
    with rt.Context([I.rt_box(4, 2, nsteps=2)], precision=rt.RT_FP64) as ctx:
        assert ctx.n == 1
