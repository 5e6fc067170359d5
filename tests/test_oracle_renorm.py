"""Pins of the optional per-step renormalisation (the remark that follows Eq. sp_en: each qpwf is
re-normalised at the end of a time step).

1. With it, every state has a^3 sum(|u|^2 + |v|^2) = 1 to rounding after each step, while the
   plain ABM lets the norms drift at its truncation level (visible at dt = 0.02).
2. It only removes that drift: the renormalised trajectory stays within the truncation level of
   the plain one (relative difference of the states about the plain norm drift).
"""
import numpy as np

from oracle import oracle as O
from paper_2009_00745_b300 import workloads as W

from .helpers import oracle_params


def run(w, steps, renormalize):
    s = O.Solver(oracle_params(w, renormalize=renormalize))
    s.set_state(w.initial_state(), 0.0, w.dt)
    norms = []
    for _ in range(steps):
        s.step(1)
        x = s.state()
        norms.append(np.sum(np.abs(x) ** 2, axis=(1, 2, 3, 4)) * w.a ** 3)
    return s.state(), np.array(norms)


def test_renormalisation_keeps_unit_norms():
    w = W.ufg_plane_waves(8, 20, noise_eps=0.3)
    w.dt = 0.02
    x0, n0 = run(w, 12, False)
    x1, n1 = run(w, 12, True)
    drift = np.max(np.abs(n0 - 1))
    assert drift > 1e-10                      # the plain ABM does drift here
    assert np.max(np.abs(n1 - 1)) < 2e-15     # renormalised: unit norms to rounding
    diff = np.linalg.norm(x1 - x0) / np.linalg.norm(x0)
    assert diff < 10 * drift                  # and otherwise the same trajectory
