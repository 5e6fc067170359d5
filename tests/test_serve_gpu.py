"""Serving loop (lise_server_*): admission under an HBM budget, overlapping
requests, and results that are the same alone and in the mix."""
import numpy as np
import pytest

from paper_2009_00745_b300 import lise as L
from paper_2009_00745_b300 import workloads as W

pytestmark = pytest.mark.gpu


def alone(w, steps, precision):
    with L.Context.from_workload(w, precision=precision) as ctx:
        ctx.set_state(w.initial_state(), 0.0, w.dt)
        ctx.step(steps)
        return ctx.state(), ctx.energy()


def test_results_identical_alone_and_in_the_mix():
    reqs = [
        (W.ufg_plane_waves(16, 40, noise_eps=0.05), 12, "fp64"),
        (W.trap_vortex(16, 24), 9, "mixed"),
        (W.ufg_plane_waves(12, 30, noise_eps=0.1), 15, "mixed"),
        (W.driven(24, 20, precision="fp64"), 7, "fp64"),
        (W.ufg_plane_waves(8, 50, noise_eps=0.2), 20, "fp64"),
        (W.ufg_plane_waves(16, 64, noise_eps=0.05), 10, "mixed"),
    ]
    refs = [alone(w, k, prec) for w, k, prec in reqs]
    fps = [L.footprint_bytes(w.nx, w.n_qp, precision=prec) for w, _, prec in reqs]
    budget = int(2.2 * max(fps))  # forces queueing: at most a few requests fit at once
    with L.Server(budget, max_active=4, steps_per_turn=3) as srv:
        ids = [srv.submit_workload(w, n_steps=k, precision=prec) for w, k, prec in reqs]
        outs = [srv.wait(i) for i in ids]
        st = srv.stats()
    assert st["peak_used_bytes"] <= budget
    assert st["peak_active"] >= 2  # requests overlapped
    for (psi, info), (ref_psi, (E, N)), (w, k, _) in zip(outs, refs, reqs):
        assert info["status"] == L.OK
        assert info["submit_s"] <= info["admit_s"] <= info["done_s"]
        assert info["t"] == pytest.approx((3 + k) * w.dt)
        assert np.array_equal(psi, ref_psi)
        assert info["E"] == E and info["N"] == N


def test_request_larger_than_budget_is_rejected():
    w = W.ufg_plane_waves(16, 64)
    fp = L.footprint_bytes(16, 64)
    with L.Server(fp // 2) as srv:
        with pytest.raises(L.LiseError) as e:
            srv.submit_workload(w, n_steps=1)
        assert e.value.status == L.ENOMEM
