"""y-slab decomposition of one instance (host index logic), on CPU ranks.

Each gloo rank holds its slab of rows plus two halo rows per neighbour,
advances it with the oracle's stage function, refreshes the halos from its
neighbours before every RK stage, and takes dt from the minimum over ranks of
its own rows' crossing times. The owned rows, gathered, must equal the
whole-domain oracle run bit for bit, and so must the dt sequence: PLM + HLLC
+ the update read two rows on each side, which the halos hold.

The reverse sweep on slabs: every rank keeps each step's input state with
eight halo rows, applies the oracle's reverse of one step to its held rows and
refreshes the cotangent halos; the gathered gradient must equal the
whole-domain oracle gradient.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import rt_inputs as I
from paper_2608_04085_b300.slabs import HALO, STEP_REVERSE_HALO, slab, slab_rows


def test_slab_rows_partition_and_halos():
    for ny, world in ((24, 1), (24, 2), (25, 3), (7, 3), (4, 2), (100, 7)):
        rows = slab_rows(ny, world)
        assert rows[0][0] == 0 and rows[-1][1] == ny
        assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
        h = [b - a for a, b in rows]
        assert max(h) - min(h) <= 1 and min(h) >= HALO
        for r in range(world):
            s = slab(ny, world, r)
            assert (s.down is None) == (r == 0) and (s.up is None) == (r == world - 1)
            assert s.e0 == (s.y0 - HALO if r > 0 else 0) and s.e1 == (s.y1 + HALO if r < world - 1 else ny)
            held = np.arange(s.e0, s.e1)
            assert list(held[s.own]) == list(range(s.y0, s.y1))
            if s.down is not None:
                below = slab(ny, world, r - 1)
                # my lower halo is exactly the rows the rank below sends up
                assert list(held[s.recv_down()]) == list(np.arange(below.e0, below.e1)[below.send_up()])
            if s.up is not None:
                above = slab(ny, world, r + 1)
                assert list(held[s.recv_up()]) == list(np.arange(above.e0, above.e1)[above.send_down()])
    assert slab(24, 3, 1, STEP_REVERSE_HALO) == slab(24, 3, 1).__class__(1, 3, 8, 16, 0, 24, 0, 2, 8)
    with pytest.raises(ValueError):
        slab_rows(5, 3)
    with pytest.raises(ValueError):
        slab(20, 3, 0, STEP_REVERSE_HALO)
    with pytest.raises(ValueError):
        slab(24, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload(cfg):
    # spacing 1/32 in x and y, so that every slab's grid has exactly the same dx, dy
    base = dict(nx=8, ny=24, x0=0.0, x1=0.25, y0=0.0, y1=0.75, y_int=0.375, y_ref=0.375, nsteps=12)
    return I.rt_box(**(base | cfg))


def _exchange(A, s, nx):
    """Refresh the halo rows of the held array A (4, held rows, nx) of slab s
    from its neighbours' owned rows."""
    import torch
    import torch.distributed as dist
    reqs, bufs = [], {}
    for nb, send, key in ((s.down, s.send_down(), "down"), (s.up, s.send_up(), "up")):
        if nb is None:
            continue
        reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(A[:, send])), nb))
        bufs[key] = torch.empty((4, s.halo, nx), dtype=torch.float64)
        reqs.append(dist.irecv(bufs[key], nb))
    for q in reqs:
        q.wait()
    if "down" in bufs:
        A[:, s.recv_down()] = bufs["down"].numpy()
    if "up" in bufs:
        A[:, s.recv_up()] = bufs["up"].numpy()


def _worker(rank, world, port, cfg, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    w = _workload(cfg)
    v = oracle.scale_to_budget(w, I.gaussian_field(3, 2, w.ny, w.nx), 1e-3)
    U = oracle.inject(w, v)
    s = slab(w.ny, world, rank)
    dy = (w.y1 - w.y0) / w.ny
    rows = lambda a, b: w.replace(ny=b - a, y0=w.y0 + a * dy, y1=w.y0 + b * dy)
    w_ext, w_own = rows(s.e0, s.e1), rows(s.y0, s.y1)
    X = np.ascontiguousarray(U[:, s.e0:s.e1])
    dts = []
    for _ in range(w.nsteps):
        wmin = torch.tensor([oracle.cfl_wmin(w_own, X[:, s.own])], dtype=torch.float64)
        dist.all_reduce(wmin, op=dist.ReduceOp.MIN)
        dt = w.cfl * float(wmin[0])
        X1 = oracle.stage(w_ext, X, dt)
        _exchange(X1, s, w.nx)
        X2 = oracle.stage(w_ext, X1, dt, base=X)
        _exchange(X2, s, w.nx)
        X = X2
        dts.append(dt)
    ke = torch.tensor([oracle.kinetic_energy(w_own, X[:, s.own])], dtype=torch.float64)
    dist.all_reduce(ke)
    out[rank] = (X[:, s.own].copy(), dts, float(ke[0]))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,cfg", [
    (2, {}),
    (3, dict(bc_y=I.BC_HYDROSTATIC, limiter=I.LIM_MC, flux=I.FLUX_HYBRID, flux_theta=1.0001)),
])
def test_slab_ranks_reproduce_the_whole_domain_bitwise(world, cfg):
    import oracle
    oracle.build()
    w = _workload(cfg)
    ref = oracle.forward(w, oracle.scale_to_budget(w, I.gaussian_field(3, 2, w.ny, w.nx), 1e-3))
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, cfg, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(180)
            assert p.exitcode == 0
        parts = [out[r] for r in range(world)]
    U = np.concatenate([p[0] for p in parts], axis=1)
    assert np.array_equal(U, ref["U"])
    for p in parts:
        assert p[1] == list(ref["dt"])
        assert p[2] == pytest.approx(ref["J_ke"], rel=1e-13)


def _grad_worker(rank, world, port, cfg, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    w = _workload(cfg)
    v = oracle.scale_to_budget(w, I.gaussian_field(3, 2, w.ny, w.nx), 1e-3)
    U = oracle.inject(w, v)
    s2, s8 = slab(w.ny, world, rank), slab(w.ny, world, rank, STEP_REVERSE_HALO)
    assert (s2.y0, s2.y1) == (s8.y0, s8.y1)
    dx, dy = oracle.grid_spacing(w)
    rows = lambda a, b: w.replace(ny=b - a, y0=w.y0 + a * dy, y1=w.y0 + b * dy)
    w2, w8, w_own = rows(s2.e0, s2.e1), rows(s8.e0, s8.e1), rows(s2.y0, s2.y1)
    held8 = lambda: np.zeros((4, s8.e1 - s8.e0, w.nx))
    # forward on halo-2 slabs; each step's input state kept with 8-row halos
    X = np.ascontiguousarray(U[:, s2.e0:s2.e1])
    states, dts = [], []
    for _ in range(w.nsteps):
        S = held8()
        S[:, s8.own] = X[:, s2.own]
        _exchange(S, s8, w.nx)
        states.append(S)
        wmin = torch.tensor([oracle.cfl_wmin(w_own, X[:, s2.own])], dtype=torch.float64)
        dist.all_reduce(wmin, op=dist.ReduceOp.MIN)
        dt = w.cfl * float(wmin[0])
        X1 = oracle.stage(w2, X, dt)
        _exchange(X1, s2, w.nx)
        X = oracle.stage(w2, X1, dt, base=X)
        _exchange(X, s2, w.nx)
        dts.append(dt)
    # terminal cotangent of J_KE = sum |m|^2 / (2 rho) dA on the owned rows
    Uo = X[:, s2.own]
    u, vy = Uo[1] / Uo[0], Uo[2] / Uo[0]
    L = held8()
    L[:, s8.own] = dx * dy * np.stack([-0.5 * (u * u + vy * vy), u, vy, 0.0 * u])
    _exchange(L, s8, w.nx)
    # reverse sweep, one step at a time
    for n in reversed(range(w.nsteps)):
        Ln = oracle.step_vjp(w8, states[n], dts[n], L)
        L = held8()
        L[:, s8.own] = Ln[:, s8.own]
        _exchange(L, s8, w.nx)
    # gradient with respect to v: rho0 (lam_m + v lam_E)
    rho0 = oracle.base_state(w)[0][s8.y0:s8.y1, None]
    lo, vo = L[:, s8.own], v[:, s8.y0:s8.y1]
    out[rank] = np.stack([rho0 * (lo[1] + vo[0] * lo[3]), rho0 * (lo[2] + vo[1] * lo[3])])
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,cfg", [
    (2, {}),
    (3, dict(bc_y=I.BC_HYDROSTATIC, limiter=I.LIM_MC, flux=I.FLUX_HYBRID, flux_theta=1.0001)),
])
def test_slab_ranks_reproduce_the_whole_domain_gradient(world, cfg):
    import oracle
    oracle.build()
    w = _workload(cfg)
    v = oracle.scale_to_budget(w, I.gaussian_field(3, 2, w.ny, w.nx), 1e-3)
    _, g_ref = oracle.gradient(w, v, oracle.forward(w, v)["dt"])
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_grad_worker, args=(r, world, port, cfg, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(180)
            assert p.exitcode == 0
        g = np.concatenate([out[r] for r in range(world)], axis=1)
    assert np.max(np.abs(g - g_ref)) <= 1e-13 * np.max(np.abs(g_ref))
