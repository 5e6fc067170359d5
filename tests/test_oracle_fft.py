"""Pins of the oracle's DFT and spectral operators (no GPU).

- The recursive mixed-radix DFT against a brute-force O(N^2) sum written from
  the forward/inverse definitions of Sec. "Discretization" (the FFT pair with
  an unnormalised forward and a 1/N inverse), and against numpy's pocketfft.
- The spectral Laplacian on plane waves: -(alpha/2) lap e^{ik.r} =
  (alpha/2) k^2 e^{ik.r} with the k grid of Sec. "Discretization", Nyquist
  mode included (zeroing applies to odd derivatives only).
- The BdG apply on a plane-wave pair reduces to the 2x2 matrix
  [[xi, Delta], [Delta*, -xi]] of Eq. tdslda.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2009_00745_b300 import workloads as W


def brute_dft(x, sign):
    n = x.size
    j = np.arange(n)
    M = np.exp(sign * 2j * np.pi * np.outer(j, j) / n)
    return M @ x


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 15, 16, 24, 25, 27, 30])
@pytest.mark.parametrize("sign", [-1, +1])
def test_dft1d_brute(n, sign):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = brute_dft(x, sign)
    got = O.dft1d(x, sign)
    assert np.linalg.norm(got - ref) <= 1e-14 * max(np.linalg.norm(ref), 1e-300) * max(1, np.log2(n))


@pytest.mark.parametrize("n", [16, 24, 32, 40, 48, 64, 80, 96])
def test_dft1d_pocketfft(n):
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = np.fft.fft(x)
    got = O.dft1d(x, -1)
    assert np.linalg.norm(got - ref) <= 1e-14 * np.linalg.norm(ref)


@pytest.mark.parametrize("shape", [(2, 3, 4), (4, 4, 4), (5, 6, 3), (6, 10, 12), (8, 8, 8), (3, 5, 2)])
def test_fft3d_brute(shape):
    rng = np.random.default_rng(sum(shape))
    v = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    nz, ny, nx = shape
    ref = v.copy()
    for axis, n in ((2, nx), (1, ny), (0, nz)):
        j = np.arange(n)
        M = np.exp(-2j * np.pi * np.outer(j, j) / n)
        ref = np.moveaxis(np.tensordot(M, np.moveaxis(ref, axis, 0), axes=(1, 0)), 0, axis)
    got = O.fft3d(v, -1)
    assert np.linalg.norm(got - ref) <= 1e-14 * np.linalg.norm(ref)
    back = O.fft3d(got, +1)
    assert np.linalg.norm(back - v) <= 1e-14 * np.linalg.norm(v)


@pytest.mark.parametrize("n", [16, 24, 32, 40, 48])
def test_fft3d_pocketfft(n):
    shape = (n, n, n) if n <= 24 else (4, 6, n)
    rng = np.random.default_rng(n)
    v = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    got = O.fft3d(v, -1)
    ref = np.fft.fftn(v)
    assert np.linalg.norm(got - ref) <= 1e-14 * np.linalg.norm(ref)
    assert np.linalg.norm(O.fft3d(v, +1) - np.fft.ifftn(v)) <= 1e-14 * np.linalg.norm(np.fft.ifftn(v))


@pytest.mark.parametrize("n,a", [(8, 1.0), (12, 0.7), (16, 1.0), (10, 1.3)])
def test_kgrid(n, a):
    # Sec. "Discretization": k_n = 2 pi n / L over the DVR range n = -N/2 .. N/2-1, stored at
    # index n mod N.  This is numpy's fftfreq times 2 pi, with the Nyquist entry at -pi/a.
    L = n * a
    expect = [2 * np.pi * (i if i < n // 2 else i - n) / L for i in range(n)]
    assert np.allclose(expect, 2 * np.pi * np.fft.fftfreq(n, d=a), rtol=0, atol=1e-15)
    assert len(set(np.round(expect, 12))) == n  # a full set of distinct momenta
    for i in range(n):
        assert O.kgrid(i, n, a) == pytest.approx(expect[i], abs=1e-15)


@pytest.mark.parametrize("modes", [[(1, 0, 0), (0, -2, 3), (-4, -4, -4), (3, 1, -2)]])
def test_laplacian_plane_waves(modes):
    nx, ny, nz, a, alpha = 8, 8, 8, 0.9, 1.7
    p = O.Params(nx, ny, nz, a=a, n_qp=1, alpha=alpha)
    for m in modes:
        pw = W.plane_wave(m, nx, ny, nz)
        k2 = sum(W.k_of_mode(mi, n, a) ** 2 for mi, n in zip(m, (nx, ny, nz)))
        got = O.kinetic(p, pw)
        ref = 0.5 * alpha * k2 * pw
        assert np.abs(got - ref).max() <= 1e-13 * max(1.0, 0.5 * alpha * k2)


def test_laplacian_nyquist_value():
    # mode -N/2 in every direction: k^2 = 3 (pi/a)^2 exactly; the Nyquist term is kept
    n, a = 6, 1.0
    p = O.Params(n, n, n, a=a, n_qp=1, alpha=1.0)
    pw = W.plane_wave((-3, -3, -3), n, n, n)
    got = O.kinetic(p, pw)
    assert np.abs(got - 0.5 * 3 * np.pi ** 2 * pw).max() < 1e-13


def test_laplacian_second_difference_limit():
    # a Gaussian well inside the box and well resolved by the grid matches its analytic
    # Laplacian to spectral accuracy
    n, a = 48, 0.35
    p = O.Params(n, n, n, a=a, n_qp=1, alpha=2.0)
    c = (np.arange(n) - n / 2) * a
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    s = 1.1
    r2 = X ** 2 + Y ** 2 + Z ** 2
    f = np.exp(-r2 / (2 * s * s)) + 0j
    lap = f * (r2 / s ** 4 - 3 / s ** 2)
    got = O.kinetic(p, f)  # = -(alpha/2) lap with alpha = 2
    assert np.abs(got + lap).max() < 1e-9


def test_apply_h_plane_wave_pair():
    nx = ny = nz = 6
    a, alpha = 1.0, 1.0
    W0, D0 = 0.37, 0.2 - 0.45j
    p = O.Params(nx, ny, nz, a=a, n_qp=2, alpha=alpha)
    rng = np.random.default_rng(3)
    psi = np.zeros(p.shape, dtype=np.complex128)
    amps = []
    for q, m in enumerate([(1, -2, 0), (3, 3, -3)]):
        pw = W.plane_wave(m, nx, ny, nz)
        U, V = rng.standard_normal(2) + 1j * rng.standard_normal(2)
        psi[q, 0], psi[q, 1] = U * pw, V * pw
        k2 = sum(W.k_of_mode(mi, n, a) ** 2 for mi, n in zip(m, (nx, ny, nz)))
        amps.append((U, V, 0.5 * alpha * k2 + W0, pw))
    Wf = np.full(p.grid, W0)
    Df = np.full(p.grid, D0, dtype=np.complex128)
    hpsi = O.apply_h(p, Wf, Df, psi)
    for q, (U, V, xi, pw) in enumerate(amps):
        hu = xi * U + D0 * V
        hv = np.conj(D0) * U - xi * V
        assert np.abs(hpsi[q, 0] - hu * pw).max() < 1e-13
        assert np.abs(hpsi[q, 1] - hv * pw).max() < 1e-13


def test_apply_h_minus_h_star_on_complex_potential_structure():
    # -h* v = -conj(h conj(v)): for a real W and the real spectral T this is -(T + W) v for
    # any complex v (T commutes with conjugation because k^2 is even in k).
    n = 6
    p = O.Params(n, n, n, a=1.0, n_qp=1, alpha=1.3)
    rng = np.random.default_rng(5)
    psi = rng.standard_normal(p.shape) + 1j * rng.standard_normal(p.shape)
    Wf = rng.standard_normal(p.grid)
    Df = np.zeros(p.grid, dtype=np.complex128)
    hpsi = O.apply_h(p, Wf, Df, psi)
    v = psi[0, 1]
    tv = np.fft.ifftn(np.fft.fftn(v) * 0.5 * 1.3 * (
        (2 * np.pi * np.fft.fftfreq(n))[:, None, None] ** 2 +
        (2 * np.pi * np.fft.fftfreq(n))[None, :, None] ** 2 +
        (2 * np.pi * np.fft.fftfreq(n))[None, None, :] ** 2))
    assert np.abs(hpsi[0, 1] + tv + Wf * v).max() < 1e-12


def test_densities_plane_waves():
    w = W.ufg_plane_waves(6, 10, noise_eps=0.0)
    p = O.Params(6, 6, 6, a=1.0, n_qp=10)
    psi = w.initial_state()
    n, nu = O.densities(p, psi)
    V = w.nxyz * w.a ** 3
    U_, V_ = w.amps[:, 0], w.amps[:, 1]
    assert np.allclose(n, 2 * np.sum(V_ ** 2) / V, rtol=1e-14, atol=0)
    assert np.allclose(nu, np.sum(U_ * V_) / V, rtol=1e-14, atol=0)
    # normalisation sum_r a^3 (|u|^2 + |v|^2) = 1 per state
    norms = np.sum(np.abs(psi) ** 2, axis=(1, 2, 3, 4)) * w.a ** 3
    assert np.allclose(norms, 1.0, rtol=0, atol=1e-14)


def test_energy_plane_waves_closed_form():
    w = W.ufg_plane_waves(6, 12, noise_eps=0.0, g=0.8, beta=-0.5)
    p = O.Params(6, 6, 6, a=1.0, n_qp=12, alpha=w.alpha, beta=w.beta, mu=w.mu, g=w.g)
    E, N = O.energy_of(p, w.initial_state(), 0.0)
    Vol = w.nxyz * w.a ** 3
    U_, V_ = w.amps[:, 0], w.amps[:, 1]
    k2 = np.array([sum(W.k_of_mode(mi, 6, 1.0) ** 2 for mi in m) for m in w.modes])
    n0 = 2 * np.sum(V_ ** 2) / Vol
    nu0 = np.sum(U_ * V_) / Vol
    Ekin = 2 * np.sum(0.5 * w.alpha * k2 * V_ ** 2)
    Eint = Vol * 0.3 * w.beta * (3 * np.pi ** 2) ** (2 / 3) * n0 ** (5 / 3)
    Epair = +w.g * nu0 ** 2 * Vol  # Eq. pairing: + g_eff |kappa|^2
    assert E == pytest.approx(Ekin + Eint + Epair, rel=1e-13, abs=1e-13)
    assert N == pytest.approx(2 * np.sum(V_ ** 2), rel=1e-14)


def test_potentials_definition():
    n = 4
    p = O.Params(n, n, n, a=1.0, n_qp=1, beta=-0.5, mu=0.3, g=1.2, drive_A=0.01, drive_Omega=0.3,
                 v_static=np.arange(n ** 3, dtype=float).reshape(n, n, n) * 1e-3)
    rng = np.random.default_rng(1)
    dens = rng.uniform(0.01, 0.2, p.grid)
    nu = rng.standard_normal(p.grid) + 1j * rng.standard_normal(p.grid)
    t = 0.7
    Wf, Df = O.potentials(p, dens, nu, t)
    zc = (np.arange(n) - n // 2)[:, None, None] * 1.0
    ref = -0.25 * (3 * np.pi ** 2 * dens) ** (2 / 3) - 0.3 + p.v_static + 0.01 * np.sin(0.3 * t) * zc
    assert np.allclose(Wf, ref, rtol=1e-14, atol=1e-15)
    assert np.allclose(Df, -1.2 * nu, rtol=1e-15, atol=0)
