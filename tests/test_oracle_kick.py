"""Pins of the oracle's boost (Eq. kick, Sec. "External boosts and external potentials").

1. Free particles (beta = g = 0, V = 0): a plane-wave pair evolves by exact phases; a kick
   chi = q.r with a lattice momentum q moves u to k + q and v to k' - q, after which the phases
   follow the new momenta.  The closed form pins the signs of the gauge factors, the restart of
   the history through the series start and the time bookkeeping.
2. A constant chi = theta is a global gauge transformation: by the definitions of the
   densities (Eqs. rho_t, nu_t) n is unchanged and nu turns by exp(2 i theta).
"""
import numpy as np

from oracle import oracle as O


def plane(N, a, m):
    x = np.arange(N) * a
    kz, ky, kx = (2 * np.pi * mm / (N * a) for mm in m)
    return np.exp(1j * (kz * x[:, None, None] + ky * x[None, :, None] + kx * x[None, None, :])), (kz, ky, kx)


def test_kick_free_particle_closed_form():
    N, a, alpha, mu, dt = 8, 1.0, 1.0, 0.3, 0.005
    m_u, m_v, m_q = (1, 0, 2), (0, -1, 1), (1, 1, 0)
    u0, ku = plane(N, a, m_u)
    v0, kv = plane(N, a, m_v)
    _, kq = plane(N, a, m_q)
    psi = np.zeros((1, 2, N, N, N), complex)
    psi[0, 0], psi[0, 1] = u0, v0
    psi /= np.sqrt(np.sum(np.abs(psi) ** 2) * a ** 3)
    p = O.Params(N, N, N, a=a, n_qp=1, alpha=alpha, beta=0.0, mu=mu, g=0.0)
    s = O.Solver(p)
    s.set_state(psi, 0.0, dt)
    s.step(4)
    t1 = s.t
    x = np.arange(N) * a
    chi = kq[0] * x[:, None, None] + kq[1] * x[None, :, None] + kq[2] * x[None, None, :]
    s.kick(chi)
    s.step(5)
    t = s.t
    assert abs(t - (t1 + 8 * dt)) < 1e-14  # 3 series steps + 5 ABM steps after the kick

    def e(k):
        return 0.5 * alpha * sum(kk * kk for kk in k) - mu

    ku2 = tuple(k + q for k, q in zip(ku, kq))
    kv2 = tuple(k - q for k, q in zip(kv, kq))
    u_exact = psi[0, 0] * np.exp(-1j * e(ku) * t1) * np.exp(1j * chi) * np.exp(-1j * e(ku2) * (t - t1))
    v_exact = psi[0, 1] * np.exp(1j * e(kv) * t1) * np.exp(-1j * chi) * np.exp(1j * e(kv2) * (t - t1))
    got = s.state()
    err = max(np.max(np.abs(got[0, 0] - u_exact)), np.max(np.abs(got[0, 1] - v_exact))) / np.max(np.abs(psi))
    assert err < 1e-9, err


def test_constant_kick_is_a_gauge_rotation():
    N, n_qp = 6, 4
    rng = np.random.default_rng(3)
    psi = rng.standard_normal((n_qp, 2, N, N, N)) + 1j * rng.standard_normal((n_qp, 2, N, N, N))
    p = O.Params(N, N, N, n_qp=n_qp)
    theta = 0.37
    k = O.kick(p, psi, np.full((N, N, N), theta))
    n0, nu0 = O.densities(p, psi)
    n1, nu1 = O.densities(p, k)
    assert np.allclose(n1, n0, rtol=1e-14, atol=0)
    assert np.allclose(nu1, nu0 * np.exp(2j * theta), rtol=1e-13, atol=1e-15)
    # and it changes nothing else: the moduli of u and v are kept element by element
    assert np.allclose(np.abs(k), np.abs(psi), rtol=1e-15)
