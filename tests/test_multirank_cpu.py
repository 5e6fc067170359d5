"""Multi-rank bench logic on CPU with the gloo backend (world size 2).

bench.py runs one independent replica per GPU under torchrun; the job time is the
maximum of the ranks' timed regions and the reported value is the units of all
ranks divided by it.  Two CPU ranks with different timings check that every rank
sees the same maximum and the same whole-job value.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 100.0 + 50.0 * rank
    value, ms = bench.whole_job_value(ms_local, units_per_rank=1e9, world=world, device="cpu")
    q.put((rank, value, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for rank, value, ms in out:
        assert ms == pytest.approx(150.0)
        assert value == pytest.approx(2 * 1e9 / 0.150)


def test_single_rank_value():
    import bench
    v, ms = bench.whole_job_value(200.0, 4e9, 1)
    assert ms == 200.0 and v == pytest.approx(2e10)
