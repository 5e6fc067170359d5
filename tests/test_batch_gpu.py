"""Batched evolutions (lise_batch_*): contexts of different lattices, state counts, step
sizes and drives stepped together in shared launches (one per kernel class and lattice
size, from a device work table; 4-step CUDA graphs) give every evolution bit for bit the
result of stepping its own context alone -- the same kernels with the same arguments."""
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


def _members():
    # (lattice, states, drive amplitude, dt): uneven sizes, two evolutions sharing a lattice
    spec = [(16, 13, 0.0, 0.005), (24, 40, 0.03, 0.005), (16, 70, 0.05, 0.004), (32, 9, 0.02, 0.005),
            (12, 5, 0.0, 0.006)]
    out = []
    for N, q, A, dt in spec:
        w = W.driven(N, q, A=A, Omega=0.3, noise_eps=0.05, steps=0)
        w.dt = dt
        out.append(w)
    return out


def _alone(w, precision, steps):
    with L.Context.from_workload(w, precision=precision) as c:
        c.set_state(w.initial_state(), 0.0, w.dt)
        c.step(steps)
        return c.state(), c.t, c.energy()


@pytest.mark.parametrize("precision", ["mixed", "mixed_strict"])
def test_batch_matches_each_context_alone(precision):
    ws = _members()
    ctxs = [L.Context.from_workload(w, precision=precision) for w in ws]
    try:
        for c, w in zip(ctxs, ws):
            c.set_state(w.initial_state(), 0.0, w.dt)
        with L.Batch(ctxs) as b:
            b.step(9)           # two 4-step graph replays and one plain step
            b.step(2)           # plain steps from another history phase
            b.sync()
        for c in ctxs:          # members continue on their own afterwards
            c.step(3)
        got = [(c.state(), c.t, c.energy()) for c in ctxs]
    finally:
        for c in ctxs:
            c.close()
    for w, g in zip(ws, got):
        ref = _alone(w, precision, 14)
        assert g[1] == ref[1]
        assert np.array_equal(g[0], ref[0]), (w.nx, w.n_qp)
        assert g[2] == ref[2]


def test_batch_argument_checks():
    w = W.ufg_plane_waves(16, 8)
    with L.Context.from_workload(w, precision="fp64") as f, L.Context.from_workload(w, precision="mixed") as m, \
            L.Context.from_workload(w, precision="mixed") as m2:
        with pytest.raises(L.LiseError) as e:        # FP64 contexts are not batched
            L.Batch([f])
        assert e.value.status == L.EINVAL
        with pytest.raises(L.LiseError) as e:        # no state yet
            L.Batch([m])
        assert e.value.status == L.ESTATE
        m.set_state(w.initial_state(), 0.0, w.dt)
        m2.set_state(w.initial_state(), 0.0, w.dt)
        with pytest.raises(L.LiseError) as e:        # the same context twice
            L.Batch([m, m])
        assert e.value.status == L.EINVAL
        b = L.Batch([m, m2])
        b.step(1)
        b.sync()
        m.step(1)                                   # moved on outside the batch
        with pytest.raises(L.LiseError) as e:
            b.step(1)
        assert e.value.status == L.ESTATE
        b.close()
