"""Pins of the external potential V_ext(r, t) and of the times at which the oracle
evaluates it (Sec. "External boosts and external potentials", Eq. tdslda; the start
procedure and Eqs. p, m, c, y of Sec. TDSLDA "Time evolution").

With alpha = beta = g = 0 the Hamiltonian is diagonal at every site (h = V_ext - mu,
Delta = 0), so every site rotates exactly:
    u(r, t) = u(r, t0) exp(-i Phi(r, t)),   v(r, t) = v(r, t0) exp(+i Phi(r, t)),
    Phi(r, t) = int_{t0}^{t} (V_ext(r, s) - mu) ds
              = (v_static(r) - mu)(t - t0) + A z_c (cos(Omega t0) - cos(Omega t)) / Omega,
with z_c = (i_z - N/2) a measured from the box centre (coordinate-dependent quantities
are taken relative to the centre, Sec. "Discretization").  Against this closed form:

  - a static potential: the whole integrator (series start + ABM) converges with
    global order 5 under dt halving;
  - one series-start step from t: its phase error is the midpoint-rule remainder
    -(dt^3/24) d^2V/dt^2 at t + dt/2, i.e. the corrector Hamiltonian is taken at
    t + dt/2 (the left end point t would leave an error of order dt^2);
  - ABM steps from an exact history: global order 5, which fails if either right-hand
    side of a step is evaluated at t_n instead of t_{n+1} (order 1);
  - a whole driven run: the phase error is the sum of the three start-step remainders
    (the ABM part is of higher order), which fails for a wrong origin of z_c, a wrong
    sign or frequency of the drive, or any wrong evaluation time.
"""
import numpy as np
import pytest

from oracle import oracle as O

from .helpers import random_state

N = 8
A, OMEGA, MU = 0.3, 2.0, 0.1


def z_c(N, a=1.0):
    return ((np.arange(N) - N // 2) * a)[:, None, None] * np.ones((1, N, N))


def phase(t0, t, vs=None, A=A, Omega=OMEGA, mu=MU, N=N):
    """Phi(r, t) of the module docstring, shape (N, N, N)."""
    ph = -mu * (t - t0) * np.ones((N, N, N))
    if vs is not None:
        ph = ph + vs * (t - t0)
    if A:
        ph = ph + A * z_c(N) * (np.cos(Omega * t0) - np.cos(Omega * t)) / Omega
    return ph


def exact(psi0, t0, t, **kw):
    ph = phase(t0, t, **kw)
    out = psi0.copy()
    out[:, 0] *= np.exp(-1j * ph)
    out[:, 1] *= np.exp(+1j * ph)
    return out


def params(n_qp, vs=None, A=A, Omega=OMEGA, mu=MU):
    return O.Params(N, N, N, a=1.0, n_qp=n_qp, alpha=0.0, beta=0.0, mu=mu, g=0.0, v_static=vs,
                    drive_A=A, drive_Omega=Omega)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def slopes(errs):
    return [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def test_static_potential_closed_form_and_order():
    # a static V: the integrator (series start + ABM) against exp(-i (V - mu) t) per site
    vs = np.random.default_rng(3).uniform(-1.0, 1.0, (N, N, N))
    psi0 = random_state(N, 3, seed=5)
    p = params(3, vs=vs, A=0.0)
    T, errs = 1.2, []
    for dt in (0.04, 0.02, 0.01):
        s = O.Solver(p)
        s.set_state(psi0, 0.0, dt)
        s.step(int(round(T / dt)) - 3)
        assert s.t == pytest.approx(T, abs=1e-12)
        errs.append(rel(s.state(), exact(psi0, 0.0, T, vs=vs, A=0.0)))
    assert errs[-1] < 1e-9, errs
    for k in slopes(errs):
        assert 4.4 < k < 5.8, (errs, slopes(errs))


@pytest.mark.parametrize("t", [0.4, 1.3])
def test_series_step_phase_error_is_the_midpoint_remainder(t):
    psi0 = random_state(N, 2, seed=7)
    p = params(2)
    zc = z_c(N)
    errs = []
    for dt in (0.04, 0.02, 0.01):
        out = O.series_step(p, psi0, t, dt)
        ex = exact(psi0, t, t + dt)
        errs.append(rel(out, ex))
        # measured phase error of u, -(Phi_mid - Phi_exact), against the midpoint-rule
        # remainder: Phi_mid - Phi_exact = -(dt^3/24) V''(t + dt/2) + O(dt^5),
        # V'' = -A Omega^2 sin(Omega t) z_c
        meas = np.angle(out[:, 0] / ex[:, 0])
        rem = -(dt ** 3 / 24.0) * (-A * OMEGA ** 2 * np.sin(OMEGA * (t + 0.5 * dt)) * zc)
        pred = -rem
        assert np.max(np.abs(meas - pred[None])) < 0.03 * np.max(np.abs(pred)), dt
        # v rotates the other way
        meas_v = np.angle(out[:, 1] / ex[:, 1])
        assert np.max(np.abs(meas_v + pred[None])) < 0.03 * np.max(np.abs(pred)), dt
    for k in slopes(errs):
        assert 2.8 < k < 3.2, (errs, slopes(errs))


def exact_history(psi0, t0, tn, dt, **kw):
    """y_n, y_{n-1} and y'_{n-k} = f(t_{n-k}, y(t_{n-k})) of the exact solution."""
    y = {k: exact(psi0, t0, tn - k * dt, **kw) for k in range(4)}
    d = []
    for k in range(4):
        tk = tn - k * dt
        w = (z_c(N) * A * np.sin(OMEGA * tk) if kw.get("A", A) else 0.0) - MU
        f = y[k].copy()
        f[:, 0] *= -1j * w     # i du/dt = (V - mu) u
        f[:, 1] *= +1j * w     # i dv/dt = -(V - mu) v
        d.append(f)
    return y[0], y[1], d


def test_abm_steps_from_exact_history_order_five():
    # Eqs. p, m, c, y alone (no series start): global order 5 only if both right-hand
    # sides of a step see V_ext at t_{n+1}
    psi0 = random_state(N, 2, seed=9)
    p = params(2)
    t0, tn, T = 0.0, 0.5, 1.5
    errs = []
    for dt in (0.04, 0.02, 0.01):
        yn, ynm1, d = exact_history(psi0, t0, tn, dt)
        s = O.Solver(p)
        s.set_history(yn, ynm1, d, tn, dt)
        s.step(int(round((T - tn) / dt)))
        assert s.t == pytest.approx(T, abs=1e-12)
        errs.append(rel(s.state(), exact(psi0, t0, T)))
    assert errs[-1] < 1e-9, errs
    for k in slopes(errs):
        assert 4.4 < k < 5.8, (errs, slopes(errs))


def test_whole_driven_run_error_is_set_by_the_start():
    # series start (3 steps) + ABM from t0 = 0.2.  The start leaves phase errors
    # delta_k (sums of the midpoint remainders r_0..r_{k-1}) on y_1..y_3; the ABM carries
    # them along (its averaging (y_n + y_{n-1})/2 keeps (2 delta_3 + delta_2)/3, about
    # 0.9 delta_3 here) and adds errors of higher order.  So the error converges with
    # order 3 and has the spatial shape and size of delta_3.
    psi0 = random_state(N, 2, seed=13)
    p = params(2)
    t0, T = 0.2, 1.2
    errs, meas = [], None
    for dt in (0.02, 0.01):
        s = O.Solver(p)
        s.set_state(psi0, t0, dt)
        s.step(int(round((T - t0) / dt)) - 3)
        ex = exact(psi0, t0, T)
        errs.append(rel(s.state(), ex))
        meas = np.angle(s.state()[:, 0] / ex[:, 0])
    assert 2.7 < slopes(errs)[0] < 3.3, errs
    dt = 0.01
    delta3 = sum(-(dt ** 3 / 24.0) * A * OMEGA ** 2 * np.sin(OMEGA * (t0 + (k + 0.5) * dt)) * z_c(N)
                 for k in range(3))
    d3 = np.broadcast_to(delta3, meas.shape)
    c = np.sum(meas * d3) / np.sum(d3 * d3)
    assert 0.8 < c < 0.98, c
    assert np.linalg.norm(meas - c * d3) < 0.05 * np.linalg.norm(c * d3)
    # z_c is measured from the box centre: the plane z = N/2 carries no drive phase
    assert np.max(np.abs(meas[:, N // 2])) < 1e-9
