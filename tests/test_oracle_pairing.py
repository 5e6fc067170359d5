"""Pins of the pairing-coupling options of the oracle.

- Eq. geff_3D: the printed lattice constant K (tests/golden) equals its integral
  definition, and the oracle's coupling obeys 1/g_eff - 1/g0 = -(m*/(4 pi^2)) (pi/a) K
  with K from that integral and m* = 1/alpha (hbar = 1).
- Eq. g0: g0(n) = g (1 - alpha_p n / n0), and d g_eff / dn matches a finite difference.
- With a density-dependent coupling the mean field gains d g_eff/dn |nu|^2 (E_pair =
  g_eff(n) |nu|^2 of Eq. pairing); the energy of a complete set of states is then
  conserved by the dynamics (a missing or wrong term breaks this by orders of magnitude).
"""
import os

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import oracle as O
from paper_2009_00745_b300 import workloads as W

from .test_oracle_dynamics import params_of, run

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "geff_lattice_constant.txt")


def golden_K():
    for line in open(GOLDEN):
        if line.startswith("K "):
            return float(line.split()[1])
    raise AssertionError("K missing")


def K_integral():
    val, err = quad(lambda th: np.log(1.0 + 1.0 / np.cos(th) ** 2), 0.0, np.pi / 4, epsabs=1e-15, epsrel=1e-15)
    return 12.0 / np.pi * val


def test_printed_K_matches_its_definition():
    assert golden_K() == pytest.approx(K_integral(), rel=1e-14)


@pytest.mark.parametrize("g0,a,alpha", [(-1.3, 1.0, 1.0), (-0.4, 0.8, 1.7), (0.2, 1.2, 0.9)])
def test_lattice_renormalisation(g0, a, alpha):
    p = O.Params(4, 4, 4, a=a, alpha=alpha, g=g0, pair_lattice=True)
    geff, dg = O.geff(p, 0.37)
    expect = 1.0 / g0 - (1.0 / alpha) / (4 * np.pi ** 2) * (np.pi / a) * K_integral()
    assert 1.0 / geff == pytest.approx(expect, rel=1e-13)
    assert dg == 0.0  # constant g0


def test_density_dependent_coupling():
    p = O.Params(4, 4, 4, g=-1.1, pair_alpha=0.5, pair_n0=0.2)
    for n in (0.0, 0.05, 0.2, 0.31):
        geff, dg = O.geff(p, n)
        assert geff == pytest.approx(-1.1 * (1 - 0.5 * n / 0.2), rel=1e-14)
    pl = p.with_(pair_lattice=True)
    n, h = 0.13, 1e-6
    gp, _ = O.geff(pl, n + h)
    gm, _ = O.geff(pl, n - h)
    _, dg = O.geff(pl, n)
    assert dg == pytest.approx((gp - gm) / (2 * h), rel=1e-8)


def test_defaults_unchanged():
    w = W.ufg_plane_waves(8, 12, noise_eps=0.1)
    p = params_of(w)
    a = run(p, w.initial_state(), 0.005, 6)
    b = run(p.with_(pair_alpha=0.0, pair_lattice=False, pair_n0=0.3), w.initial_state(), 0.005, 6)
    assert np.array_equal(a.state(), b.state())


def test_energy_conserved_with_density_dependent_renormalised_pairing():
    n = 6
    w = W.ufg_plane_waves(n, n ** 3, noise_eps=0.3, beta=-0.5, g=-0.8)
    n0 = 2 * np.sum(w.amps[:, 1] ** 2) / (w.nxyz * w.a ** 3)
    p = params_of(w, pair_alpha=0.6, pair_n0=n0, pair_lattice=True)
    psi0 = w.initial_state()
    E0, N0 = O.energy_of(p, psi0, 0.0)
    drift = []
    for dt in (0.01, 0.005):
        s = run(p, psi0, dt, int(round(0.6 / dt)))
        drift.append(abs(s.energy()[0] - E0) / abs(E0))
    assert drift[1] < 1e-8, drift
    assert drift[1] < drift[0] / 8, drift
    # and the coupling really varies: Delta is not -g nu
    nn, nu = O.densities(p, psi0)
    Wp, Dp = O.potentials(p, nn, nu, 0.0)
    assert np.abs(Dp + p.g * nu).max() > 1e-3 * np.abs(p.g * nu).max()
