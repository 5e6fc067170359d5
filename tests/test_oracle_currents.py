"""Pins of the oracle's first derivative and current density (Eq. j; Sec. "Discretization": odd
derivatives drop the Nyquist coefficient).

1. Plane waves: d/dx e^{i q x} = i q e^{i q x} exactly below the Nyquist index; the Nyquist mode
   itself has derivative 0 (the dropped coefficient).
2. The derivative of a real function is real (the reason for dropping the coefficient).
3. Current of plane-wave states: v = A e^{i q.r} carries j = -2 q |A|^2 (spin factor 2; the
   v component is the time-reversed partner, so its momentum counts with a minus sign).
4. Galilean boost: a kick chi = p.r (Eq. kick) adds p n(r) to the current, for band-limited states.
"""
import numpy as np

from oracle import oracle as O

from .helpers import random_state


def grid_x(N, a):
    return np.arange(N) * a


def test_gradient_plane_waves_and_nyquist():
    N, a = 8, 0.7
    p = O.Params(N, N, N, a=a)
    x = grid_x(N, a)
    L = N * a
    for axis, shape in ((0, (1, 1, N)), (1, (1, N, 1)), (2, (N, 1, 1))):
        for m in (1, -3, 2):
            q = 2 * np.pi * m / L
            f = np.broadcast_to(np.exp(1j * q * x).reshape(shape), (N, N, N)).copy()
            g = O.gradient(p, f, axis)
            assert np.max(np.abs(g - 1j * q * f)) < 1e-13
        f = np.broadcast_to(np.cos(np.pi * x / a).reshape(shape), (N, N, N)).astype(complex)  # Nyquist mode
        assert np.max(np.abs(O.gradient(p, f, axis))) < 1e-13


def test_gradient_of_real_field_is_real():
    N = 12
    p = O.Params(N, N, N)
    f = np.random.default_rng(5).standard_normal((N, N, N)).astype(complex)
    for axis in range(3):
        assert np.max(np.abs(O.gradient(p, f, axis).imag)) < 1e-13


def test_plane_wave_current():
    N, a = 8, 1.0
    L = N * a
    x = grid_x(N, a)
    ms = [(1, 0, -1), (0, 2, 1)]
    amps = [0.3, 0.7]
    psi = np.zeros((2, 2, N, N, N), complex)
    expect = np.zeros(3)
    for s, (m, A) in enumerate(zip(ms, amps)):
        qx, qy, qz = (2 * np.pi * mm / L for mm in m)
        psi[s, 1] = A * np.exp(1j * (qx * x[None, None, :] + qy * x[None, :, None] + qz * x[:, None, None]))
        psi[s, 0] = 0.5  # u does not enter j
        expect += -2 * np.array([qx, qy, qz]) * A * A
    j = O.currents(O.Params(N, N, N, a=a, n_qp=2), psi)
    for c in range(3):
        assert np.max(np.abs(j[c] - expect[c])) < 1e-13


def test_boost_adds_p_times_density():
    N, n_qp = 12, 5
    psi = random_state(N, n_qp, seed=8, kmax=3)  # band-limited: no Nyquist involvement
    p = O.Params(N, N, N, n_qp=n_qp)
    x = grid_x(N, 1.0)
    pv = 2 * np.pi * np.array([1, -1, 2]) / N  # lattice momentum (x, y, z)
    chi = pv[0] * x[None, None, :] + pv[1] * x[None, :, None] + pv[2] * x[:, None, None]
    j0 = O.currents(p, psi)
    j1 = O.currents(p, O.kick(p, psi, chi))
    n, _ = O.densities(p, psi)
    for c in range(3):
        assert np.max(np.abs(j1[c] - j0[c] - pv[c] * n)) < 1e-12 * max(1.0, np.max(np.abs(n)))
