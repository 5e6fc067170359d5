"""Exchanges for sharded densities (lise_set_shard in include/lise.h).

One evolution's states are split over ranks (a context per rank, one GPU each in a real
run).  Before every density reduction the library hands the exchange its block of
partial sums, [3][n_groups_all][N^3] doubles (n, Re nu, Im nu), with this rank's groups
filled in; the exchange fills in every other rank's groups.  This is the paper's
structure (Sec. "CPU-GPU hybrid structure": partial densities on each GPU, a global
reduction, the full densities back on every GPU).  Every rank's groups are copied as
they are (broadcasts, no arithmetic), so each rank then reduces all groups in the
global order exactly as a single context holding every state would.

host_exchange   torch.distributed with CPU tensors (gloo) on the library's pinned host
                copy of the block (lise_shard.on_device = 0).
device_exchange the same on the device block (e.g. NCCL), enqueued on the context's
                stream (lise_shard.on_device = 1).

Argument marshalling only: the reductions themselves run in the library's kernels.
"""
import ctypes as C

import numpy as np


def _rank_ranges(first, n_local, group, device):
    import torch
    import torch.distributed as dist
    mine = torch.tensor([first, n_local], dtype=torch.int64, device=device)
    every = [torch.zeros(2, dtype=torch.int64, device=device) for _ in range(dist.get_world_size(group))]
    dist.all_gather(every, mine, group=group)
    out = [(int(x[0]), int(x[1])) for x in every]
    groups = sorted(g for f, n in out for g in range(f, f + n))
    if groups != list(range(len(groups))) or len(set(groups)) != len(groups):
        raise ValueError(f"the ranks' group ranges {out} do not tile 0..n_groups_all-1")
    return out


def _broadcast_groups(t, ranges, group):
    import torch.distributed as dist
    for idx, (f, n) in enumerate(ranges):
        src = idx if group is None else dist.get_global_rank(group, idx)
        for k in range(3):
            dist.broadcast(t[k, f:f + n], src=src, group=group)


def host_exchange(group=None):
    """Exchange on the host copy (lise_shard.on_device = 0) over torch.distributed (gloo)."""
    state = {}

    def exchange(parts, on_device, stream, nxyz, first, n_local, n_all):
        import torch
        if on_device:
            raise ValueError("host_exchange works on the host copy (on_device = 0)")
        n = 3 * n_all * nxyz
        a = np.ctypeslib.as_array((C.c_double * n).from_address(parts)).reshape(3, n_all, nxyz)
        if "ranges" not in state:
            state["ranges"] = _rank_ranges(first, n_local, group, "cpu")
            if sum(nl for _, nl in state["ranges"]) != n_all:
                raise ValueError("n_groups_all differs from the sum of the ranks' groups")
        _broadcast_groups(torch.from_numpy(a), state["ranges"], group)

    return exchange


class _DeviceBlock:
    def __init__(self, ptr, count):
        self.__cuda_array_interface__ = {"shape": (count,), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def device_exchange(group=None):
    """Exchange on the device block (lise_shard.on_device = 1) over torch.distributed (NCCL),
    enqueued on the context's stream."""
    state = {}

    def exchange(parts, on_device, stream, nxyz, first, n_local, n_all):
        import torch
        if not on_device:
            raise ValueError("device_exchange works on the device block (on_device = 1)")
        t = torch.as_tensor(_DeviceBlock(parts, 3 * n_all * nxyz), device="cuda").view(3, n_all, nxyz)
        with torch.cuda.stream(torch.cuda.ExternalStream(int(stream))):
            if "ranges" not in state:
                state["ranges"] = _rank_ranges(first, n_local, group, "cuda")
            _broadcast_groups(t, state["ranges"], group)

    return exchange
