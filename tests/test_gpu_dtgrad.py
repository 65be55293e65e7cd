"""Gradient through the CFL step control on the GPU (rt_gradient with
RT_GRAD_DT) against the oracle's reverse sweep that differentiates the same
control (dt_n = cfl * min crossing time, shared among tied candidates; a
horizon-clipped last step dt = T - t)."""
import numpy as np
import pytest

import rt_inputs as I

pytestmark = pytest.mark.gpu


def _cases():
    return [I.rt_box(16, 32, nsteps=20), I.rt_box(16, 48, T=0.1, limiter=I.LIM_NONE),
            I.paper_unit_square(16, 0.05), I.rt_box(12, 40, T=0.08, limiter=I.LIM_MC, ncomp=I.PERT_VY)]


def _starts(ws):
    import oracle
    return [oracle.scale_to_budget(w, I.gaussian_field(60 + k, w.ncomp, w.ny, w.nx), 1e-3).ravel()
            for k, w in enumerate(ws)]


@pytest.mark.parametrize("ckpt", ["store_all", "sqrt", "revolve"])
def test_dt_gradient_fp64_matches_oracle(ckpt):
    """FP64, uneven batch, every checkpoint plan: relative L2 error <= 1e-10
    against the oracle (the GPU forms dU^{n+1}/d dt from stage differences,
    U1 - U^n, which costs a few digits against the oracle's forward-mode
    derivative), and the frozen-dt gradient differs by far more."""
    import oracle
    import paper_2608_04085_b300 as rt
    ws = _cases()
    vs = _starts(ws)
    mode = {"store_all": rt.RT_CKPT_STORE_ALL, "sqrt": rt.RT_CKPT_SQRT, "revolve": rt.RT_CKPT_REVOLVE}[ckpt]
    slot = 4 * 8 * sum(w.nx * w.ny for w in ws)
    cap = 6 * slot if ckpt == "revolve" else 0.0
    with rt.Context(ws, precision=rt.RT_FP64, ckpt=mode, ckpt_cap_bytes=cap) as ctx:
        J, g, st = ctx.gradient(np.concatenate(vs), dt_grad=True)
        _, gf, _ = ctx.gradient(np.concatenate(vs))
        offs, sizes = ctx.offsets, ctx.sizes
    if ckpt == "revolve":
        assert st["segments"] < 0
    for k, w in enumerate(ws):
        ek0 = oracle.baseline_ek(w) if w.objective == I.OBJ_EK_ANOMALY_L2 else None
        Jr, gr, _ = oracle.gradient_dt(w, vs[k].reshape(w.ncomp, w.ny, w.nx), ek0)
        gk = g[offs[k]:offs[k] + sizes[k]]
        assert J[k] == pytest.approx(Jr, rel=1e-13)
        err = np.linalg.norm(gk - gr.ravel()) / np.linalg.norm(gr)
        assert err <= 1e-10, (k, err)
        frozen = np.linalg.norm(gf[offs[k]:offs[k] + sizes[k]] - gr.ravel()) / np.linalg.norm(gr)
        assert frozen > 100 * max(err, 1e-14), (k, frozen)


def test_dt_gradient_matches_gpu_central_differences_and_fp32():
    """Central differences of the GPU forward run with its own step control
    agree with the FP64 dt gradient to 1e-6; the FP32 dt gradient has cosine
    >= 0.999 with it."""
    import paper_2608_04085_b300 as rt
    w = I.rt_box(32, 96, T=0.2, limiter=I.LIM_NONE)
    v = _starts([w])[0]
    with rt.Context([w], precision=rt.RT_FP64) as ctx:
        _, g, _ = ctx.gradient(v, dt_grad=True)
        for k in range(3):
            d = I.gaussian_field(500 + k, 2, w.ny, w.nx).ravel()
            h = 1e-6 * np.linalg.norm(v) / np.linalg.norm(d)
            Jp = ctx.forward(v + h * d)[0][0]
            Jm = ctx.forward(v - h * d)[0][0]
            fd = (Jp - Jm) / (2 * h)
            assert g @ d == pytest.approx(fd, rel=1e-6)
    with rt.Context([w], precision=rt.RT_FP32_STATE) as c32:
        _, g32, _ = c32.gradient(v, dt_grad=True)
    cos = (g32 @ g) / (np.linalg.norm(g32) * np.linalg.norm(g))
    assert cos >= 0.999, cos


def test_dt_gradient_drives_the_cnop():
    """cnop_solve with RT_GRAD_DT runs the L-BFGS on the dt-differentiated
    gradient; J rises and the iterate stays on the budget."""
    import oracle
    import paper_2608_04085_b300 as rt
    w = I.rt_box(16, 32, nsteps=15)
    xi = I.gaussian_field(9, 2, w.ny, w.nx).ravel()
    with rt.Context([w], precision=rt.RT_FP64) as ctx:
        v, J, res = ctx.cnop(xi, 1e-4, 3, dt_grad=True)
    assert res["status"] == rt.RT_OK and res["iterations"] == 3
    assert res["J_history"][-1, 0] > res["J_history"][0, 0]
    assert oracle.constraint(w, v) == pytest.approx(1e-4, rel=1e-12)
