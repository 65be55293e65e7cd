"""The batched and long-horizon workload shapes, at shortened horizons.

- Uneven batch: 64 instances (32 x 128x384, 24 x 256x768, 8 x 512x1536), each
  from its own seeded start with delta cycling 1e-5, 1e-4, 1e-3, advance in
  one launch per stage; sampled instances of every grid equal their
  single-instance runs bitwise (FP32 state), forward and gradient.
- 1024x3072 grid, FP32 state: a memory cap that forces binomial (revolve)
  checkpointing gives the same gradient, bitwise, as sqrt(N) checkpointing.
"""
import numpy as np
import pytest

import rt_inputs as I

pytestmark = pytest.mark.gpu


def _uneven(T):
    grids = [(128, 384)] * 32 + [(256, 768)] * 24 + [(512, 1536)] * 8
    return [I.rt_box(nx, ny, T=T) for nx, ny in grids]


def test_uneven_batch_equals_single_instances():
    import paper_2608_04085_b300 as rt
    ws = _uneven(0.05)
    deltas = [1e-5, 1e-4, 1e-3]
    xi = [I.gaussian_field(i, 2, w.ny, w.nx).ravel() for i, w in enumerate(ws)]
    eps = [deltas[i % 3] for i in range(len(ws))]
    # one stage-kernel variant for both runs: FP32 FMA contraction may differ between variants
    tile = rt.RT_STAGE_TILE
    with rt.Context(ws, precision=rt.RT_FP32_STATE, ckpt=rt.RT_CKPT_SQRT, stage_kernel=tile) as ctx:
        v = ctx.project(np.concatenate(xi), eps, to_budget=True)
        J, _, st = ctx.forward(v)
        Jg, g, stg = ctx.gradient(v)
        offs, sizes = ctx.offsets, ctx.sizes
        states = {i: ctx.state(i) for i in (0, 40, 63)}
    assert stg["segments"] > 1
    for i in (0, 40, 63):
        vi = v[offs[i]:offs[i] + sizes[i]]
        with rt.Context([ws[i]], precision=rt.RT_FP32_STATE, ckpt=rt.RT_CKPT_SQRT, stage_kernel=tile) as c1:
            J1, _, _ = c1.forward(vi)
            assert J1[0] == J[i]
            assert np.array_equal(c1.state(0), states[i])
            Jg1, g1, _ = c1.gradient(vi)
        assert Jg1[0] == Jg[i]
        assert np.array_equal(g1, g[offs[i]:offs[i] + sizes[i]])


def test_large_grid_revolve_equals_sqrt():
    import paper_2608_04085_b300 as rt
    w = I.rt_box(1024, 3072, T=0.01)
    v = None
    out = {}
    slot = 4 * 4 * w.nx * w.ny
    for mode, cap in ((rt.RT_CKPT_SQRT, 0.0), (rt.RT_CKPT_REVOLVE, 10 * slot)):
        with rt.Context([w], precision=rt.RT_FP32_STATE, ckpt=mode, ckpt_cap_bytes=cap,
                        stage_kernel=rt.RT_STAGE_TILE) as ctx:
            if v is None:
                v = ctx.project(I.gaussian_field(5, 2, w.ny, w.nx).ravel(), 1e-4, to_budget=True)
            J, g, st = ctx.gradient(v)
            out[mode] = (J[0], g, st)
    assert out[rt.RT_CKPT_REVOLVE][2]["segments"] < 0  # revolve reports recomputed steps
    assert out[rt.RT_CKPT_SQRT][0] == out[rt.RT_CKPT_REVOLVE][0]
    assert np.array_equal(out[rt.RT_CKPT_SQRT][1], out[rt.RT_CKPT_REVOLVE][1])


def test_fma_peak_is_plausible():
    """The FMA microbenchmark: FP32 between 20 and 150 TFLOP/s (148 SMs x
    128 lanes x 2 FLOPs at 1-2.1 GHz is 38-80), FP64 well below FP32."""
    import paper_2608_04085_b300 as rt
    f32, f64 = rt.fma_peak()
    assert 20.0 < f32 < 150.0, f32
    assert 0.05 < f64 < f32, (f32, f64)
