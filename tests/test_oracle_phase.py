"""Pins of the trivial-phase removal (Eq. sp_en): i dpsi_k/dt = (H - eta_k) psi_k with
eta_k = <psi_k|H|psi_k>.  The removed phase exp(-i int eta_k dt) commutes with the
dynamics (densities are invariant under a phase per state), so:

- a self-consistent stationary BCS state (H psi_k = E_k psi_k) does not move at all;
- free particles (H constant, eta_k conserved) follow the closed form times e^{i eta_k t};
- densities agree with the unmodified evolution to the integrator's truncation level.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2009_00745_b300 import workloads as W

from .test_oracle_dynamics import free_exact, free_setup, params_of, rel, run, stationary_setup


def test_eta_of_stationary_state_is_the_quasiparticle_energy():
    w, p, Ek = stationary_setup()
    psi = w.initial_state()
    n, nu = O.densities(p, psi)
    Wp, Dp = O.potentials(p, n, nu, 0.0)
    eta = O.eta(p, psi, O.apply_h(p, Wp, Dp, psi))
    assert np.allclose(eta, Ek, rtol=0, atol=1e-12)


def test_stationary_state_stays_put():
    w, p, Ek = stationary_setup()
    p = p.with_(remove_phase=True)
    psi0 = w.initial_state()
    s = run(p, psi0, 0.01, 60)
    assert rel(s.state(), psi0) < 1e-13


def test_free_particles_phase_removed_closed_form():
    p, psi0 = free_setup(seed=4)
    pr = p.with_(remove_phase=True)
    H = O.apply_h(p, np.full(p.grid, -p.mu), np.zeros(p.grid, complex), psi0)
    eta = O.eta(p, psi0, H)
    s = run(pr, psi0, 0.01, 80)
    exact = free_exact(p, psi0, s.t) * np.exp(1j * eta * s.t)[:, None, None, None, None]
    assert rel(s.state(), exact) < 1e-9


def test_densities_match_unremoved_evolution():
    w = W.ufg_plane_waves(8, 16, noise_eps=0.2, beta=-0.5, g=1.0)
    p = params_of(w)
    psi0 = w.initial_state()
    a = run(p, psi0, 0.005, 40)
    b = run(p.with_(remove_phase=True), psi0, 0.005, 40)
    na, nua = a.densities()
    nb, nub = b.densities()
    assert rel(nb, na) < 1e-9
    assert rel(nub, nua) < 1e-9
    # per state, the two solutions differ by a phase only
    ov = np.abs(np.einsum("qcxyz,qcxyz->q", a.state().conj(), b.state()))
    assert np.allclose(ov, np.einsum("qcxyz,qcxyz->q", a.state().conj(), a.state()).real, rtol=1e-8)
    # and the phase is really removed: the unmodified run rotates, the other does not
    assert rel(b.state(), psi0) < rel(a.state(), psi0)
