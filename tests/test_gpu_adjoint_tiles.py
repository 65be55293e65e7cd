"""Adjoint tiles of 32 x 24 cells on 384 threads (FP32 only) against tiles of
32 x 16 cells on 256 threads. Every cell sums its face contributions in the
same order in both, so the gradients agree to FP32 rounding (the compiler may
contract the two instantiations differently; measured bit for bit), for
uniform and uneven batches, y-slabs, the generic-limiter kernels and both
tile-load modes. The autotuner keeps one of the two for FP32; FP64 always
uses 16-row tiles."""
import numpy as np
import pytest

import rt_inputs as I

pytestmark = pytest.mark.gpu


def _rt():
    import paper_2608_04085_b300 as rt
    return rt


def _v(ws, seed, eps=1e-4):
    import oracle
    return np.concatenate([oracle.scale_to_budget(w, I.gaussian_field(seed + k, w.ncomp, w.ny, w.nx), eps).ravel()
                           for k, w in enumerate(ws)])


CASES = {
    "box256x192_x4": ([I.rt_box(256, 192, nsteps=40)] * 4, {}),
    "uneven_mc_hydro": ([I.rt_box(128, 96, nsteps=30), I.rt_box(100, 90, nsteps=30, limiter=I.LIM_MC,
                                                                  bc_y=I.BC_HYDROSTATIC, ncomp=I.PERT_VY),
                         I.rt_box(160, 64, nsteps=30), I.rt_box(37, 45, nsteps=30)], {}),
    "slabs3": ([I.rt_box(128, 160, nsteps=25)], {"y_slabs": 3}),
    "plain_loads": ([I.rt_box(128, 96, nsteps=30)] * 2, {"tile_loads": 1}),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp32_adjoint_24_row_tiles_equal_16_row_tiles(name, monkeypatch):
    rt = _rt()
    ws, kw = CASES[name]
    v = _v(ws, 5)
    out = {}
    for rows in (16, 24):
        monkeypatch.setenv("RT_CNOP_ADJ_ROWS", str(rows))
        with rt.Context(ws, precision=rt.RT_FP32_STATE, ckpt=rt.RT_CKPT_SQRT, **kw) as ctx:
            assert ctx.adjoint_rows()[0] == rows
            J, g, _ = ctx.gradient(v)
            out[rows] = (J, g)
    (J16, g16), (J24, g24) = out[16], out[24]
    assert np.array_equal(J16, J24)
    scale = np.max(np.abs(g16))
    assert np.max(np.abs(g24 - g16)) <= 1e-6 * scale, np.max(np.abs(g24 - g16)) / scale


def test_adjoint_tile_choice(monkeypatch):
    rt = _rt()
    ws = [I.rt_box(256, 192, nsteps=5)] * 2
    monkeypatch.delenv("RT_CNOP_ADJ_ROWS", raising=False)
    with rt.Context(ws, precision=rt.RT_FP32_STATE) as ctx:
        rows, ms = ctx.adjoint_rows()
        assert rows in (16, 24)
        assert ms[16] > 0 and ms[24] > 0
        assert ms[rows] == min(ms.values())
    monkeypatch.setenv("RT_CNOP_ADJ_ROWS", "24")
    with rt.Context(ws, precision=rt.RT_FP64) as ctx:
        assert ctx.adjoint_rows()[0] == 16
