"""Bounded device waits: a wait that runs out is reported, leaves the GPU usable, and the
context recovers through a new state.

lise_set_wait_limit(ctx, 0) makes every bounded wait give up without polling (nothing
else is changed: no fault, no trap, no endless loop).  The kernels that wait on the
hardware are the tensor-memory planes kernels (FP64 path, 32^3 and 48^3 lattices: the MMA
completion and the hand-offs between their roles) and the staged pencils kernel (mixed
path: the tensor-memory-accelerator copies); a block whose wait gave up lets the work it
has in flight finish, frees its tensor memory and exits, and the host reports LISE_ETIMEOUT
at the next synchronising call.
"""
import numpy as np
import pytest

from paper_2009_00745_b300 import lise as L
from paper_2009_00745_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2009_00745_b300 import build
    build.build()
    L.load()


@pytest.mark.parametrize("N,precision,n_qp", [(32, "fp64", 8), (48, "fp64", 4), (16, "mixed", 12), (48, "mixed", 6)])
def test_wait_that_runs_out_is_reported_and_the_context_recovers(N, precision, n_qp):
    w = W.ufg_plane_waves(N, n_qp, noise_eps=0.05)
    with L.Context.from_workload(w, precision=precision) as ref:
        ref.set_state(w.initial_state(), 0.0, w.dt)
        ref.step(6)
        expect = ref.state()
    with L.Context.from_workload(w, precision=precision) as ctx:
        ctx.set_state(w.initial_state(), 0.0, w.dt)
        ctx.set_wait_limit(0)        # every bounded wait gives up at once
        ctx.step(2)                  # plain launches
        with pytest.raises(L.LiseError) as e:
            ctx.sync()
        assert e.value.status == L.ETIMEOUT
        with pytest.raises(L.LiseError) as e:   # sticky until a new state replaces the history
            ctx.step(1)
        assert e.value.status == L.ETIMEOUT
        ctx.set_wait_limit(-1)       # back to the default bound
        ctx.set_state(w.initial_state(), 0.0, w.dt)
        ctx.step(6)                  # one graph replay of 4 steps + 2 plain steps
        got = ctx.state()
    assert np.array_equal(got, expect)


def test_timeout_inside_a_graph_replay():
    # the limit is a kernel parameter: changing it drops the captured graphs, so a replay
    # after the change gives up too, and one after restoring it does not
    w = W.ufg_plane_waves(16, 10, noise_eps=0.05)
    with L.Context.from_workload(w, precision="mixed") as ctx:
        ctx.set_state(w.initial_state(), 0.0, w.dt)
        ctx.step(4)                  # captures and replays a graph with the default bound
        ctx.sync()
        ctx.set_wait_limit(0)
        ctx.step(4)
        with pytest.raises(L.LiseError) as e:
            ctx.sync()
        assert e.value.status == L.ETIMEOUT
        ctx.set_wait_limit(-1)
        ctx.set_state(w.initial_state(), 0.0, w.dt)
        ctx.step(8)
        ctx.sync()
