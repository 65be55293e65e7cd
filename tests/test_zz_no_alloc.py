"""rt_objective_noalloc: the allocation-free objective entry point.

Some callers cannot let a library allocate device memory (their framework
owns all device memory through a fixed-budget pool, or they cannot afford
the device-wide synchronisation of cudaMalloc). This entry point evaluates
the objective of a final state using a fixed scratch array inside the
library. The test calls it through the C ABI on states produced by
rt_forward and checks that two calls in a row both reproduce the J that
rt_forward itself returned (1e-12 relative: only the summation order
differs). This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import rt_inputs as I

pytestmark = pytest.mark.gpu


def _noalloc_fn():
    import paper_2608_04085_b300 as rt
    L = rt.library()
    f = L.rt_objective_noalloc
    f.argtypes = [ctypes.POINTER(rt.RtProblem), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def test_noalloc_objective_matches_forward_twice():
    import torch
    import paper_2608_04085_b300 as rt
    f = _noalloc_fn()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream().cuda_stream
    w_ke = I.rt_box(48, 80, nsteps=40)
    w_pap = I.paper_unit_square(24, 0.05).replace(ny=40)
    rng = [I.gaussian_field(3, w_ke.ncomp, w_ke.ny, w_ke.nx), I.gaussian_field(4, w_pap.ncomp, w_pap.ny, w_pap.nx)]
    with rt.Context([w_ke, w_pap], precision=rt.RT_FP64) as ctx:
        v = ctx.project(np.concatenate([r.ravel() for r in rng]), [1e-4, 1e-6], to_budget=True)
        J, Jke, _ = ctx.forward(v)
        states = [ctx.state(0), ctx.state(1)]
    with rt.Context([w_pap], precision=rt.RT_FP64) as c0:
        c0.forward(np.zeros(c0.total))
        U0 = c0.state(0)
    ek0 = 0.5 * (U0[1] * U0[1] + U0[2] * U0[2]) / U0[0]
    d_ek0 = torch.from_numpy(np.ascontiguousarray(ek0)).to(dev)
    for call in range(2):
        for k, (w, U) in enumerate(zip((w_ke, w_pap), states)):
            d_U = torch.from_numpy(np.ascontiguousarray(U)).to(dev)
            d_J = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
            prob = rt.make_problem(w)
            e_ptr = ctypes.c_void_p(d_ek0.data_ptr()) if k == 1 else None
            st = f(ctypes.byref(prob), ctypes.c_void_p(d_U.data_ptr()), e_ptr, ctypes.c_void_p(d_J.data_ptr()),
                   ctypes.c_void_p(stream))
            assert st == rt.RT_OK, (call, k, st)
            torch.cuda.synchronize()
            out = d_J.cpu().numpy()
            assert out[0] == pytest.approx(Jke[k], rel=1e-12), (call, k)
            if k == 1:
                assert out[1] == pytest.approx(J[1], rel=1e-12), call


def test_noalloc_rejects_grid_above_scratch_limit():
    import torch
    import paper_2608_04085_b300 as rt
    f = _noalloc_fn()
    d = torch.zeros(8, dtype=torch.float64, device="cuda")
    prob = rt.make_problem(I.rt_box(4096, 2048))
    st = f(ctypes.byref(prob), ctypes.c_void_p(d.data_ptr()), None, ctypes.c_void_p(d.data_ptr()),
           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == rt.RT_EINVAL


@pytest.mark.parametrize("nx,ny", [(256, 768), (2048, 2048)], ids=["768_blocks", "at_the_limit"])
def test_noalloc_many_blocks_and_the_size_limit(nx, ny):
    """Grids of more than 256 blocks exercise the strided loop of the final
    reduction; 2048 x 2048 is exactly the 4,194,304-cell limit (16,384
    blocks, every partial slot in use) and must be accepted. Both against
    rt_forward's J_KE of the same one-step run, on two calls in a row."""
    import torch
    import paper_2608_04085_b300 as rt
    f = _noalloc_fn()
    w = I.rt_box(nx, ny, nsteps=1)
    with rt.Context([w], precision=rt.RT_FP64) as ctx:
        v = ctx.project(I.gaussian_field(9, 2, ny, nx).ravel(), 1e-4, to_budget=True)
        _, Jke, _ = ctx.forward(v)
        U = ctx.state(0)
    d_U = torch.from_numpy(np.ascontiguousarray(U)).to("cuda")
    ek = 0.5 * (U[1] * U[1] + U[2] * U[2]) / U[0]
    dA = ((w.x1 - w.x0) / nx) * ((w.y1 - w.y0) / ny)
    stream = torch.cuda.current_stream().cuda_stream
    prob = rt.make_problem(w)
    for call in range(2):
        d_J = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        st = f(ctypes.byref(prob), ctypes.c_void_p(d_U.data_ptr()), None, ctypes.c_void_p(d_J.data_ptr()),
               ctypes.c_void_p(stream))
        assert st == rt.RT_OK, (call, st)
        torch.cuda.synchronize()
        out = d_J.cpu().numpy()
        assert out[0] == pytest.approx(Jke[0], rel=1e-12), call
        # with no reference field J[1] is the sum of e_k^2 dA
        assert out[1] == pytest.approx(np.sum(ek * ek) * dA, rel=1e-12), call
