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
    a = bench.bench_inputs(0)
    b = bench.bench_inputs(1)
    assert a.shape == b.shape == (bench.BATCH * 2 * bench.NY * bench.NX,)
    assert not np.array_equal(a[:1000], b[:1000])
    assert np.array_equal(a, bench.bench_inputs(0))
