"""Serving loop (lise_server_*): admission under an HBM budget, overlapping
requests, and results that are the same alone and in the mix."""
import time

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


@pytest.mark.parametrize("batching", [False, True])
def test_results_identical_alone_and_in_the_mix(batching):
    # with batching, the mixed-precision requests are stepped together in shared launches
    # (joining and leaving the batch as they start and finish); the FP64 ones alone
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
        if batching:
            srv.set_batching(True)
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


@pytest.mark.parametrize("policy,small_first", [("fifo", False), ("first_fit", True)])
def test_admission_policy(policy, small_first):
    # A long request occupies the budget so that the big one cannot start beside it;
    # the small one fits.  FIFO keeps arrival order (small waits behind big); first fit
    # admits the small one at once.
    a = W.ufg_plane_waves(16, 96, noise_eps=0.05)
    big = W.ufg_plane_waves(16, 256, noise_eps=0.05)
    small = W.ufg_plane_waves(16, 16, noise_eps=0.05)
    fa, fb, fs = (L.footprint_bytes(16, w.n_qp) for w in (a, big, small))
    budget = fa + fb - 1
    assert fa + fs <= budget and fb <= budget
    states = [w.initial_state() for w in (a, big, small)]  # built before the clock starts
    with L.Server(budget, max_active=4, steps_per_turn=2) as srv:
        srv.set_admission(policy, max_skips=4)
        # the long request runs far longer than the two submissions that follow it
        ia = srv.submit_workload(a, psi=states[0], n_steps=1000)
        ib = srv.submit_workload(big, psi=states[1], n_steps=2)
        i_s = srv.submit_workload(small, psi=states[2], n_steps=2)
        t_end = time.time() + 120
        while not srv.poll(ia) and time.time() < t_end:
            time.sleep(0.01)
        assert srv.poll(ia)
        infos = {k: srv.wait(i, want_state=False)[1] for k, i in (("a", ia), ("big", ib), ("small", i_s))}
    assert all(v["status"] == L.OK for v in infos.values())
    assert (infos["small"]["admit_s"] < infos["big"]["admit_s"]) == small_first
    # the big request could only start after the long one had finished
    assert infos["big"]["admit_s"] >= infos["a"]["done_s"]


def test_first_fit_skip_bound():
    # with max_skips = 0 first fit never passes over a waiting request: arrival order
    a = W.ufg_plane_waves(16, 96, noise_eps=0.05)
    big = W.ufg_plane_waves(16, 256, noise_eps=0.05)
    small = W.ufg_plane_waves(16, 16, noise_eps=0.05)
    fa, fb = L.footprint_bytes(16, 96), L.footprint_bytes(16, 256)
    states = [w.initial_state() for w in (a, big, small)]
    with L.Server(fa + fb - 1, max_active=4, steps_per_turn=2) as srv:
        srv.set_admission("first_fit", max_skips=0)
        ids = [srv.submit_workload(w, psi=x, n_steps=k) for w, x, k in ((a, states[0], 1000), (big, states[1], 2),
                                                                         (small, states[2], 2))]
        infos = [srv.wait(i, want_state=False)[1] for i in ids]
    assert infos[2]["admit_s"] >= infos[1]["admit_s"]
    with L.Server(1 << 30) as srv:
        assert L.load().lise_server_set_admission(srv._h, 7, 0) == L.EINVAL
        assert L.load().lise_server_set_admission(srv._h, L.ADMIT_FIRST_FIT, -1) == L.EINVAL


def test_borrowed_submission_matches_copied():
    reqs = [(W.ufg_plane_waves(16, 40, noise_eps=0.05), 8, "fp64"), (W.trap_vortex(16, 24), 9, "mixed")]
    refs = [alone(w, k, prec) for w, k, prec in reqs]
    inputs = [w.initial_state() for w, _, _ in reqs]
    outs = [np.zeros_like(x) for x in inputs]
    with L.Server(1 << 34, max_active=2, steps_per_turn=3) as srv:
        ids = [srv.submit(w.nx, w.n_qp, x, 0.0, w.dt, k, a=w.a, alpha=w.alpha, beta=w.beta, mu=w.mu, g=w.g,
                          v_static=w.v_static, drive_A=w.drive_A, drive_Omega=w.drive_Omega, precision=prec,
                          copy=False, out=o)
               for (w, k, prec), x, o in zip(reqs, inputs, outs)]
        # no output buffer: the evolution runs, E and N come back, no state
        w0, k0, p0 = reqs[0]
        i_none = srv.submit(w0.nx, w0.n_qp, inputs[0], 0.0, w0.dt, k0, a=w0.a, alpha=w0.alpha, beta=w0.beta,
                            mu=w0.mu, g=w0.g, precision=p0, copy=False)
        got = [srv.wait(i) for i in ids]
        psi_none, info_none = srv.wait(i_none)
    for (psi, info), o, (ref_psi, (E, N)) in zip(got, outs, refs):
        assert psi is o and info["status"] == L.OK
        assert np.array_equal(o, ref_psi)
        assert info["E"] == E and info["N"] == N
    assert psi_none is None and info_none["status"] == L.OK and info_none["E"] == refs[0][1][0]


def test_batched_serving_of_mixed_requests():
    # only mixed requests, all admitted at once, uneven step counts: members leave the batch
    # as they finish and the batch is rebuilt for the rest; every result as if alone
    reqs = [(W.driven(16, 30, A=0.03, noise_eps=0.05), 6), (W.ufg_plane_waves(24, 20, noise_eps=0.05), 11),
            (W.driven(16, 12, A=0.01, noise_eps=0.05), 9), (W.trap_vortex(12, 16), 14)]
    for w, _ in reqs:
        w.precision = "mixed"
    refs = [alone(w, k, "mixed") for w, k in reqs]
    with L.Server(1 << 34, max_active=8, steps_per_turn=4) as srv:
        srv.set_batching(True)
        ids = [srv.submit_workload(w, n_steps=k) for w, k in reqs]
        outs = [srv.wait(i) for i in ids]
        with pytest.raises(L.LiseError) as e:   # only before the first submission
            srv.set_batching(False)
        assert e.value.status == L.ESTATE
    for (psi, info), (ref_psi, (E, N)) in zip(outs, refs):
        assert info["status"] == L.OK
        assert np.array_equal(psi, ref_psi)
        assert info["E"] == E
