"""CNOP optimiser on the GPU (cnop_solve) against the oracle's spectral
projected gradient (Sec. 3.4, Eq. projection).

FP64: same start on the budget sphere, same iteration rule; the iterates
agree to rounding. FP32 state: the CNOP's cosine against the FP64 CNOP from
the same start is at least 0.999 and J agrees to 1e-4.
"""
import numpy as np
import pytest

import rt_inputs as I

pytestmark = pytest.mark.gpu


def _start(w, seed, eps):
    import oracle
    return oracle.scale_to_budget(w, I.gaussian_field(seed, w.ncomp, w.ny, w.nx), eps)


def test_cnop_fp64_matches_oracle_spg():
    import oracle
    import paper_2608_04085_b300 as rt
    w = I.rt_box(16, 32, nsteps=20)
    eps = 1e-4
    v0 = _start(w, 8, eps)
    ref = oracle.spg(w, v0, eps, iters=6)
    with rt.Context([w], precision=rt.RT_FP64) as ctx:
        v, J, res = ctx.cnop(v0.ravel(), eps, 6, method=rt.RT_CNOP_SPG)
    assert res["status"] == rt.RT_OK
    assert res["iterations"] == len(ref["records"])
    assert J[0] == pytest.approx(ref["J"], rel=1e-10)
    err = np.linalg.norm(v - ref["v"].ravel()) / np.linalg.norm(ref["v"])
    assert err <= 1e-8, err
    assert oracle.constraint(w, v.reshape(v0.shape)) == pytest.approx(eps, rel=1e-12)
    assert J[0] > ref["history"][0]  # the optimiser increased J


@pytest.mark.parametrize("method", [0, 1], ids=["spg", "lbfgs"])
def test_cnop_batch_equals_single_runs(method):
    import paper_2608_04085_b300 as rt
    ws = [I.rt_box(16, 32, nsteps=15), I.rt_box(12, 40, nsteps=12, ncomp=I.PERT_VY, limiter=I.LIM_MC)]
    eps = [1e-4, 1e-3]
    starts = [_start(w, 20 + k, eps[k]).ravel() for k, w in enumerate(ws)]
    with rt.Context(ws, precision=rt.RT_FP64) as ctx:
        vb, Jb, _ = ctx.cnop(np.concatenate(starts), eps, 4, method=method)
    off = 0
    for k, w in enumerate(ws):
        with rt.Context([w], precision=rt.RT_FP64) as ctx:
            vs, Js, _ = ctx.cnop(starts[k], eps[k], 4, method=method)
        n = starts[k].size
        assert Jb[k] == pytest.approx(Js[0], rel=1e-13)
        assert np.allclose(vb[off:off + n], vs, rtol=0, atol=1e-12 * np.max(np.abs(vs)))
        off += n


def test_cnop_fp32_cosine_against_fp64():
    import paper_2608_04085_b300 as rt
    w = I.rt_box(48, 96, nsteps=0, T=0.3)
    eps = 1e-4
    v0 = _start(w, 3, eps).ravel()
    out = {}
    for prec in (rt.RT_FP64, rt.RT_FP32_STATE):
        with rt.Context([w], precision=prec) as ctx:
            out[prec] = ctx.cnop(v0, eps, 8, method=rt.RT_CNOP_SPG)
    v64, J64, _ = out[rt.RT_FP64]
    v32, J32, _ = out[rt.RT_FP32_STATE]
    cos = abs(v32 @ v64) / (np.linalg.norm(v32) * np.linalg.norm(v64))
    assert cos >= 0.999, cos
    assert abs(J32[0] - J64[0]) / J64[0] <= 1e-4


def test_cnop_localised_start_and_autograd_wrapper():
    """h_loc localises the start at the interface before scaling onto the
    budget; the torch.autograd wrapper returns the same gradient as
    rt_gradient."""
    import torch
    import oracle
    import paper_2608_04085_b300 as rt
    from paper_2608_04085_b300.autograd import objective
    w = I.rt_box(16, 48, nsteps=10)
    xi = I.gaussian_field(5, 2, w.ny, w.nx)
    with rt.Context([w], precision=rt.RT_FP64) as ctx:
        v, J, res = ctx.cnop(xi.ravel(), 1e-4, 0, h_loc=0.15)
        ref = oracle.random_start(w, xi, 0.15, 1e-4).ravel()
        assert np.linalg.norm(v - ref) / np.linalg.norm(ref) <= 1e-12
        vt = torch.from_numpy(ref).cuda().requires_grad_(True)
        Jt = objective(vt, ctx)
        Jt.sum().backward()
        _, g, _ = ctx.gradient(ref)
        assert np.allclose(vt.grad.cpu().numpy(), g, rtol=1e-14, atol=0)


def test_lbfgs_fp64_matches_oracle():
    """Projected L-BFGS (the paper's optimiser) on the GPU follows the oracle's
    iterates to rounding, on the RT box and on the paper's unit-square
    configuration (u_y only, squared e_k anomaly, eps = 1e-6, localised start)."""
    import oracle
    import paper_2608_04085_b300 as rt
    cases = [(I.rt_box(16, 32, nsteps=20), 1e-4, 0.0, 8, 6),
             (I.paper_unit_square(24, 0.08), 1e-6, 0.1, 9, 5)]
    for w, eps, h_loc, seed, iters in cases:
        xi = I.gaussian_field(seed, w.ncomp, w.ny, w.nx)
        v0 = oracle.random_start(w, xi, h_loc, eps) if h_loc > 0 else oracle.scale_to_budget(w, xi, eps)
        ek0 = oracle.baseline_ek(w) if w.objective == I.OBJ_EK_ANOMALY_L2 else None
        ref = oracle.lbfgs(w, v0, eps, iters=iters, ek0=ek0)
        with rt.Context([w], precision=rt.RT_FP64) as ctx:
            v, J, res = ctx.cnop(xi.ravel(), eps, iters, method=rt.RT_CNOP_LBFGS, h_loc=h_loc)
        assert res["status"] == rt.RT_OK
        assert res["iterations"] == len(ref["records"]) == iters
        assert res["gradient_evals"] == ref["grads"]
        assert J[0] == pytest.approx(ref["J"], rel=1e-10)
        err = np.linalg.norm(v - ref["v"].ravel()) / np.linalg.norm(ref["v"])
        assert err <= 1e-8, err
        assert oracle.constraint(w, v.reshape(v0.shape)) == pytest.approx(eps, rel=1e-12)
        assert J[0] > ref["history"][0]


def test_lbfgs_fp32_cosine_against_fp64_and_beats_spg():
    """FP32-state L-BFGS CNOP has cosine >= 0.999 with the FP64 one from the
    same start; with the same number of gradient evaluations it reaches a J
    at least as large as the spectral projected gradient's."""
    import paper_2608_04085_b300 as rt
    w = I.rt_box(48, 96, nsteps=0, T=0.3)
    eps = 1e-4
    xi = I.gaussian_field(3, 2, w.ny, w.nx).ravel()
    out = {}
    for prec in (rt.RT_FP64, rt.RT_FP32_STATE):
        with rt.Context([w], precision=prec) as ctx:
            out[prec] = ctx.cnop(xi, eps, 8, method=rt.RT_CNOP_LBFGS)
        with rt.Context([w], precision=prec) as ctx:
            out[(prec, "spg")] = ctx.cnop(xi, eps, 8, method=rt.RT_CNOP_SPG)
    v64, J64, r64 = out[rt.RT_FP64]
    v32, J32, _ = out[rt.RT_FP32_STATE]
    cos = abs(v32 @ v64) / (np.linalg.norm(v32) * np.linalg.norm(v64))
    assert cos >= 0.999, cos
    assert abs(J32[0] - J64[0]) / J64[0] <= 1e-4
    _, Jspg, rspg = out[(rt.RT_FP64, "spg")]
    assert r64["gradient_evals"] == rspg["gradient_evals"]
    assert J64[0] >= Jspg[0] * (1 - 1e-12), (J64[0], Jspg[0])


def test_cnop_rejects_bad_arguments():
    import paper_2608_04085_b300 as rt
    w = I.rt_box(16, 32, nsteps=5)
    with rt.Context([w], precision=rt.RT_FP64) as ctx:
        for method in (rt.RT_CNOP_SPG, rt.RT_CNOP_LBFGS):
            with pytest.raises(RuntimeError, match="C = 0"):
                ctx.cnop(np.zeros(2 * w.nx * w.ny), 1e-4, 2, method=method)
        with pytest.raises(RuntimeError, match="unknown CNOP method"):
            ctx.cnop(I.gaussian_field(1, 2, w.ny, w.nx).ravel(), 1e-4, 2, method=7)
        # the context stays usable, with every instance switched back on
        J, _, _ = ctx.forward(np.zeros(2 * w.nx * w.ny))
        assert np.isfinite(J[0])
