"""Sharded densities on the GPU: one evolution's states split over two processes (one
context each, both on cuda:0), partial density sums exchanged through the host with
gloo before every reduction (lise_set_shard, paper_2009_00745_b300/shard.py), against
one context holding all states with the same density group size: the states, densities
and energy must agree bit for bit (every group is summed in the same order, the groups
are reduced in their global order).

The two processes never wait on each other on the device: each finishes its kernels,
copies its partial sums to the host and meets the other rank in gloo.
"""
import os
import socket
import tempfile

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu

GROUP = 4


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload(precision, n_qp=24, N=16):
    from paper_2009_00745_b300 import workloads as W
    w = W.driven(N, n_qp, A=0.05, noise_eps=0.05, steps=9)
    w.precision = precision
    return w


def _run(ctx, w, psi, path):
    ctx.set_state(psi, 0.0, w.dt)
    ctx.step(w.steps)
    n, nu = ctx.densities()
    E, Np = ctx.energy()
    j = ctx.currents()
    np.savez(path, psi=ctx.state(), n=n, nu=nu, E=E, N=Np, j=j)


def _rank_main(rank, world, port, precision, split, outdir):
    import sys
    import torch
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_2009_00745_b300 import lise as L
    from paper_2009_00745_b300 import shard
    w = _workload(precision)
    q0, q1 = split[rank], split[rank + 1]
    psi = w.initial_state(q0, q1)
    n_all = -(-w.n_qp // GROUP)
    with L.Context(w.nx, q1 - q0, a=w.a, alpha=w.alpha, beta=w.beta, mu=w.mu, g=w.g, drive_A=w.drive_A,
                   drive_Omega=w.drive_Omega, precision=precision) as ctx:
        ctx.set_shard(GROUP, first_group=q0 // GROUP, n_groups_all=n_all, exchange=shard.host_exchange())
        _run(ctx, w, psi, os.path.join(outdir, f"rank{rank}.npz"))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("precision,split", [("fp64", (0, 12, 24)), ("mixed", (0, 16, 24))])
def test_two_shards_match_one_context_bitwise(precision, split):
    from paper_2009_00745_b300 import build
    from paper_2009_00745_b300 import lise as L
    build.build()
    w = _workload(precision)
    with tempfile.TemporaryDirectory() as d:
        port = _free_port()
        ctx = mp.get_context("spawn")
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, precision, split, d)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=600)
            assert p.exitcode == 0
        parts = [dict(np.load(os.path.join(d, f"rank{r}.npz"))) for r in range(2)]
        with L.Context.from_workload(w, precision=precision) as one:
            one.set_shard(GROUP)  # same group size, no other shard
            _run(one, w, w.initial_state(), os.path.join(d, "one.npz"))
        ref = dict(np.load(os.path.join(d, "one.npz")))
    assert np.array_equal(np.concatenate([parts[0]["psi"], parts[1]["psi"]]), ref["psi"])
    for r in range(2):
        for k in ("n", "nu", "E", "N", "j"):
            assert np.array_equal(parts[r][k], ref[k]), (r, k)


def test_set_shard_argument_checks():
    from paper_2009_00745_b300 import lise as L
    with L.Context(8, 10) as ctx:
        for kw in (dict(group_size=0), dict(group_size=65), dict(group_size=4, first_group=-1),
                   dict(group_size=4, first_group=0, n_groups_all=2)):   # 10 states need 3 groups of 4
            with pytest.raises(L.LiseError) as e:
                ctx.set_shard(**kw)
            assert e.value.status == L.EINVAL
        ctx.set_shard(4, first_group=1, n_groups_all=4)
        # an exchange that fails is reported, not ignored
        def bad(*a):
            raise RuntimeError("peer lost")
        ctx.set_shard(5, first_group=0, n_groups_all=2, exchange=bad)
        from paper_2009_00745_b300 import workloads as W
        w = W.ufg_plane_waves(8, 10)
        with pytest.raises(L.LiseError) as e:
            ctx.set_state(w.initial_state(), 0.0, w.dt)
        assert e.value.status == L.EEXCHANGE
