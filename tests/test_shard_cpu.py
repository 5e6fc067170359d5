"""Sharded densities, host side (no GPU): the exchange of paper_2009_00745_b300/shard.py
between two gloo ranks on CPU, on blocks laid out as the library hands them over
([3][n_groups_all][N^3] doubles, this rank's groups filled in), and the ctypes callback
marshalling of Context.set_shard (an exception becomes a non-zero return).

The paper sums the partial densities of every GPU's states with a global reduction
before the potentials are built (Sec. "CPU-GPU hybrid structure"); here every rank
receives the other ranks' groups unchanged, so each can reduce all groups in the global
order (bit-for-bit the single-context sum).
"""
import ctypes as C
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _block(n_all, nxyz):
    """The full block every rank must end with: distinct values per (array, group, site)."""
    return (np.arange(3 * n_all * nxyz, dtype=np.float64).reshape(3, n_all, nxyz) * 0.37 - 5.0)


def _rank_main(rank, world, port, ranges, nxyz, q):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2009_00745_b300 import shard
    n_all = sum(n for _, n in ranges)
    first, n_local = ranges[rank]
    full = _block(n_all, nxyz)
    ex = shard.host_exchange()
    ok = True
    for call in range(3):   # the ranges are gathered once, then reused
        buf = np.full((3, n_all, nxyz), np.nan)
        buf[:, first:first + n_local] = full[:, first:first + n_local] + call
        ex(buf.ctypes.data, False, None, nxyz, first, n_local, n_all)
        ok = ok and np.array_equal(buf, full + call)
    q.put((rank, ok))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("ranges", [[(0, 3), (3, 3)], [(0, 4), (4, 1)], [(2, 3), (0, 2)]])
def test_host_exchange_two_gloo_ranks(ranges):
    # even split, uneven split, and ranks whose groups are not in rank order
    world, nxyz = 2, 64
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, ranges, nxyz, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out == {0: True, 1: True}


def test_exchange_callback_marshalling():
    # the ctypes wrapper Context.set_shard installs: the Python exchange sees the block's
    # address and sizes; an exception is reported as a non-zero return (LISE_EEXCHANGE)
    from paper_2009_00745_b300 import lise as L
    seen = []

    def good(parts, on_device, stream, nxyz, first, n_local, n_all):
        seen.append((parts, on_device, stream, nxyz, first, n_local, n_all))

    def bad(*args):
        raise RuntimeError("peer lost")

    def wrap(f):  # the same wrapping as Context.set_shard
        def cb_py(user, parts, on_dev, stream, nxyz, first, nloc, nall):
            try:
                f(parts, bool(on_dev), stream, nxyz, first, nloc, nall)
                return 0
            except Exception:
                return 1
        return L.EXCHANGE_FN(cb_py)

    buf = np.zeros(3 * 2 * 8)
    g = wrap(good)
    assert g(None, buf.ctypes.data, 0, None, 8, 1, 1, 2) == 0
    assert seen == [(buf.ctypes.data, False, None, 8, 1, 1, 2)]
    assert wrap(bad)(None, buf.ctypes.data, 0, None, 8, 0, 1, 2) == 1
    sh = L._Shard(4, 0, 3, g, None, 0, 0)
    assert sh.group_size == 4 and sh.n_groups_all == 3
    assert C.cast(sh.exchange, C.c_void_p).value is not None
    assert C.cast(L._Shard(4, 0, 3, L.EXCHANGE_FN(), None, 0, 0).exchange, C.c_void_p).value is None
