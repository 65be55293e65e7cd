"""Multi-rank logic of bench.py on CPU (gloo, world size 2): every rank gets
its own seeded batch, and the timing reduction takes the max of the times and
the sum of the cell updates (weak scaling, no data-path collective)."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, cells = bench.reduce_timing(100.0 + 50.0 * rank, 1000.0 * (rank + 1), world, None)
    out[rank] = (ms, cells)
    dist.barrier()
    dist.destroy_process_group()


def test_timing_reduction_two_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(world):
            assert out[r] == (150.0, 3000.0)


def test_ranks_get_disjoint_seeded_batches():
    import bench
    a = bench.config_inputs(bench.make_config("default", 0))
    b = bench.config_inputs(bench.make_config("default", 1))
    assert a.shape == b.shape == (32 * 2 * bench.NY * bench.NX,)
    assert not np.array_equal(a[:1000], b[:1000])
    assert np.array_equal(a, bench.config_inputs(bench.make_config("default", 0)))


def test_uneven_and_high_resolution_configurations():
    """The uneven batch: 32 x 128x384, 24 x 256x768, 8 x 512x1536 in that
    order, T = 2, budgets cycling 1e-5, 1e-4, 1e-3 by instance, seed = index;
    the high-resolution case: one 1024x3072 instance, T = 6, revolve capped
    at 40 GB."""
    import bench
    c = bench.make_config("uneven64", 0)
    assert [(w.nx, w.ny) for w in c.problems] == [(128, 384)] * 32 + [(256, 768)] * 24 + [(512, 1536)] * 8
    assert {w.T for w in c.problems} == {2.0}
    assert c.deltas[:4] == [1e-5, 1e-4, 1e-3, 1e-5] and c.seeds == list(range(64))
    assert bench.make_config("uneven64", 1).seeds == list(range(64, 128))
    h = bench.make_config("hires", 0)
    assert [(w.nx, w.ny, w.T) for w in h.problems] == [(1024, 3072, 6.0)]
    assert h.cap_bytes == 40e9


def test_clock_summary_of_nvidia_smi_rows():
    """The clocks object of the JSON line: median SM clock, highest max clock,
    every throttle reason that was Active in any sample; unreadable clock
    fields are skipped."""
    import bench
    row = lambda sm, mx, *act: ["0", sm, mx, "900.0", "0x0"] + list(act)
    na, a = "Not Active", "Active"
    rows = [row("2032", "2032", na, na, na, na), row("1980", "2032", na, na, na, a),
            row("[N/A]", "2032", na, na, na, na), row("2010", "2032", na, na, na, na)]
    out = bench.summarise_clocks(rows)
    assert out == {"sm_mhz": 2010.0, "sm_max_mhz": 2032.0, "reasons": ["sw_power_cap"], "samples": 4}
    hot = bench.summarise_clocks([row("1500", "2032", a, na, a, na)])
    assert hot["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.summarise_clocks([])["reasons"] == ["no samples"]


def test_host_cpu_description():
    import bench
    h = bench.host_cpu()
    assert h["host_cpus"] == __import__("os").cpu_count() and h["host_cpus"] >= 1
    assert h["cpu_model"] is None or isinstance(h["cpu_model"], str)
