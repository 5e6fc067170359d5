"""Pins of the pairing-coupling options of the oracle.

- Eq. geff_3D: the printed lattice constant K (tests/golden) equals its integral
  definition, and the oracle's coupling obeys 1/g_eff - 1/g0 = -(m*/(4 pi^2)) (pi/a) K
  with K from that integral and m* = 1/alpha (hbar = 1).
- Eq. g0: g0(n) = g (1 - alpha_p n / n0), and d g_eff / dn matches a finite difference.
- With a density-dependent coupling the mean field gains d g_eff/dn |nu|^2 (E_pair =
  g_eff(n) |nu|^2 of Eq. pairing); the energy of a complete set of states is then
  conserved by the dynamics (a missing or wrong term breaks this by orders of magnitude).
- Eq. geff (spherical momentum cutoff E_c): the logarithmic branch (k_F^2 > 0) equals the
  principal-value integral m*/(2 pi^2) PV int_0^{k_c} k^2 dk / (k^2 - k_F^2); both branches equal
  one power series in k_F^2 (the arctan branch is the continuation of the logarithmic one);
  continuity at k_F = 0; g_eff = g0 where k_c^2 <= 0; the total d g_eff/dn (through g0(n) and
  through U(n) inside k_F, k_c) matches finite differences; and the energy of a complete set
  of states in a trap with sites on both branches is conserved.
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


# ------------------------------------------------------- Eq. geff, spherical cutoff --
# hbar = 1 and m* = 1/alpha: k_F^2 = 2 m* (mu - U), k_c^2 = 2 m* (E_c + mu - U) (Eq. geff);
# the correction is read back as c = 1/g0 - 1/g_eff.

def _cut_params(alpha=1.3, mu=0.7, ec=2.0, g=-0.9, **kw):
    return O.Params(4, 4, 4, a=1.0, alpha=alpha, mu=mu, g=g, pair_ec=ec, **kw)


def _c_of(p, u):
    geff, _ = O.geff(p, 0.2, u)
    return 1.0 / p.g - 1.0 / geff


def _kf2_kc(p, u):
    m = 1.0 / p.alpha
    kf2 = 2 * m * (p.mu - u)
    return kf2, np.sqrt(kf2 + 2 * m * p.pair_ec), m


@pytest.mark.parametrize("u", [-1.5, -0.2, 0.4, 0.69])
def test_cutoff_first_branch_is_the_principal_value_integral(u):
    # k_F^2 > 0: c = m* / (2 pi^2) PV int_0^{k_c} k^2 / (k^2 - k_F^2) dk (the spherical momentum
    # cutoff the equation is derived from), by adaptive quadrature with the Cauchy weight
    p = _cut_params()
    kf2, kc, m = _kf2_kc(p, u)
    kf = np.sqrt(kf2)
    pv, _ = quad(lambda k: k * k / (k + kf), 0.0, kc, weight="cauchy", wvar=kf, epsabs=1e-14, epsrel=1e-13)
    assert _c_of(p, u) == pytest.approx(m / (2 * np.pi ** 2) * pv, rel=1e-11)


def _series(kf2, kc, m, terms=400):
    # k_c - k_F artanh(k_F/k_c) as its power series in s = k_F^2 (|s| < k_c^2): one analytic
    # function of s on both sides of s = 0
    s = 0.0
    for j in range(terms):
        s += kf2 ** (j + 1) / ((2 * j + 1) * kc ** (2 * j + 1))
    return m / (2 * np.pi ** 2) * (kc - s)


@pytest.mark.parametrize("u", [0.4, 0.69, 0.71, 1.2, 1.5])
def test_cutoff_branches_are_one_analytic_function(u):
    # the k_F^2 < 0 branch (arctan) is the continuation of the logarithmic one in k_F^2
    p = _cut_params()
    kf2, kc, m = _kf2_kc(p, u)
    assert abs(kf2) < 0.8 * kc * kc
    assert _c_of(p, u) == pytest.approx(_series(kf2, kc, m), rel=1e-12)


def test_cutoff_continuous_at_zero_fermi_momentum():
    p = _cut_params()
    kf2, kc, m = _kf2_kc(p, p.mu)
    assert kf2 == 0.0
    c0 = _c_of(p, p.mu)
    assert c0 == pytest.approx(m * kc / (2 * np.pi ** 2), rel=1e-14)
    for h in (1e-6, -1e-6):
        assert _c_of(p, p.mu + h) == pytest.approx(c0, rel=1e-5)


def test_cutoff_empty_sphere_keeps_g0():
    # E_c + mu - U <= 0: no momenta below the cutoff, g_eff = g0 (reading)
    p = _cut_params(pair_alpha=0.4, pair_n0=0.5)
    geff, dg = O.geff(p, 0.2, p.mu + p.pair_ec + 0.1)
    assert geff == pytest.approx(p.g * (1 - 0.4 * 0.2 / 0.5), rel=1e-15)
    assert dg == pytest.approx(-p.g * 0.4 / 0.5, rel=1e-15)


@pytest.mark.parametrize("v,pair_alpha", [(-1.0, 0.0), (0.3, 0.0), (3.0, 0.0), (-1.0, 0.5), (3.0, 0.5)])
def test_cutoff_density_derivative(v, pair_alpha):
    # total d g_eff / dn at a site with static potential v: through g0(n) and through
    # U(n) = beta (3 pi^2 n)^(2/3) / 2 inside k_F and k_c
    p = _cut_params(beta=-0.7, pair_alpha=pair_alpha, pair_n0=0.6)
    U = lambda n: 0.5 * p.beta * (3 * np.pi ** 2 * n) ** (2.0 / 3.0)
    n, h = 0.35, 1e-6
    gp, _ = O.geff(p, n + h, U(n + h) + v)
    gm, _ = O.geff(p, n - h, U(n - h) + v)
    _, dg = O.geff(p, n, U(n) + v)
    kf2, _, _ = _kf2_kc(p, U(n) + v)
    assert (kf2 > 0) == (v < 2.0)
    assert dg == pytest.approx((gp - gm) / (2 * h), rel=1e-7)


def test_energy_conserved_with_spherical_cutoff_pairing():
    # a trap that puts some sites on each branch of Eq. geff; E_pair = g_eff(n, r) |nu|^2 and the
    # mean field's d g_eff/dn |nu|^2 must be consistent for the energy to be conserved
    n = 6
    w = W.ufg_plane_waves(n, n ** 3, noise_eps=0.3, beta=-0.5, g=-0.8)
    p = params_of(w, v_static=W.harmonic_trap(n, 0.6), pair_ec=4.5, mu=0.0)
    psi0 = w.initial_state()
    nn, _ = O.densities(p, psi0)
    u_loc = 0.5 * p.beta * (3 * np.pi ** 2 * nn) ** (2.0 / 3.0) + p.v_static
    assert (u_loc > p.mu).sum() > 8 and (u_loc < p.mu).sum() > 100
    E0, _ = O.energy_of(p, psi0, 0.0)
    drift = []
    for dt in (0.01, 0.005):
        s = run(p, psi0, dt, int(round(0.6 / dt)))
        drift.append(abs(s.energy()[0] - E0) / abs(E0))
    assert drift[1] < 1e-8, drift
    assert drift[1] < drift[0] / 8, drift
