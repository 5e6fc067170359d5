"""Pin of the oracle's Adams-Bashforth-Milne formulas to the error constants the
paper prints beside them (tests/golden/abm_error_constants.txt; arXiv:2009.00745,
Sec. "TDSLDA / Time evolution", Eqs. p, m, c, y).

With an exact polynomial history the formulas' errors are pure: for y = t^5 the
predictor and corrector miss y(t_{n+1}) by exactly 161/480 and -9/480 times
h^5 y^(5); for y = t^6/720 (with p_n - c_n taken from the previous step and exact
derivatives) the modifier and the final value miss by exactly 923/2880 and
-43/2880 times h^6 y^(6).  These four numbers fix every coefficient of the four
formulas, including the y'_n coefficient of Eq. p that the paper prints without
a number.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "abm_error_constants.txt")


def golden():
    out = {}
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, k, num, den = line.split()
        out[name] = (int(k), Fraction(int(num), int(den)))
    return out


def hist(y, dy, h, t0=0.0):
    """Exact history at t_n = t0: y_n, y_{n-1}, y'_n .. y'_{n-3}, as 1-element arrays
    (complex, to exercise the complex path with a phase)."""
    ph = np.exp(0.3j)
    t = lambda k: t0 - k * h
    return ([np.array([y(t(0)) * ph]), np.array([y(t(1)) * ph])],
            [np.array([dy(t(k)) * ph]) for k in range(4)], ph)


@pytest.mark.parametrize("h", [1.0, 0.5, 0.125])
def test_predictor_and_corrector_constants(h):
    G = golden()
    y = lambda t: t ** 5
    dy = lambda t: 5 * t ** 4
    (yn, ynm1), d, ph = hist(y, dy, h)
    p = O.abm_predictor(h, yn, ynm1, *d)
    exact = y(h) * ph
    k, C = G["predictor"]
    assert k == 5
    assert (exact - p[0]) == pytest.approx(float(C) * h ** 5 * 120 * ph, rel=1e-12)
    mp = np.array([dy(h) * ph])  # exact m'_{n+1}
    c = O.abm_corrector(h, yn, ynm1, mp, d[0], d[1], d[2])
    k, C = G["corrector"]
    assert k == 5
    assert (exact - c[0]) == pytest.approx(float(C) * h ** 5 * 120 * ph, rel=1e-12)


@pytest.mark.parametrize("h", [1.0, 0.5, 0.25])
def test_modifier_and_final_constants(h):
    G = golden()
    y = lambda t: t ** 6 / 720.0
    dy = lambda t: t ** 5 / 120.0
    # previous step (t_{n-1} -> t_n) gives p_n - c_n
    (yp, ypm1), dprev, ph = hist(y, dy, h, t0=-h)
    p_n = O.abm_predictor(h, yp, ypm1, *dprev)
    c_n = O.abm_corrector(h, yp, ypm1, np.array([dy(0.0) * ph]), dprev[0], dprev[1], dprev[2])
    pc_n = p_n - c_n
    (yn, ynm1), d, _ = hist(y, dy, h)
    p = O.abm_predictor(h, yn, ynm1, *d)
    m = O.abm_modifier(p, pc_n)
    exact = y(h) * ph
    k, C = G["modifier"]
    assert k == 6
    assert (exact - m[0]) == pytest.approx(float(C) * h ** 6 * ph, rel=1e-11)
    c = O.abm_corrector(h, yn, ynm1, np.array([dy(h) * ph]), d[0], d[1], d[2])
    yfin, pc = O.abm_final(p, c)
    k, C = G["final"]
    assert k == 6
    assert (exact - yfin[0]) == pytest.approx(float(C) * h ** 6 * ph, rel=1e-11)
    assert pc[0] == pytest.approx(p[0] - c[0], rel=1e-15)


def test_principal_root_amplitude_decay():
    # steady state of the whole scheme on u' = -i w u (a free plane wave): the amplitude
    # falls by (43/2880) / rho'(1) * (w h)^6 per step, rho(z) = z^2 - (z + 1)/2 being the
    # first characteristic polynomial of Eqs. p and c (rho'(1) = 3/2); Richardson
    # extrapolation removes the O((w h)^7) term.
    from paper_2009_00745_b300 import workloads as W
    G = golden()
    n = 4
    p = O.Params(n, n, n, a=1.0, n_qp=1, alpha=1.0)
    psi = np.zeros(p.shape, complex)
    pw = W.plane_wave((1, 1, 1), n, n, n) / np.sqrt(n ** 3)
    psi[0, 0] = pw
    om = 0.5 * 3 * (2 * np.pi / n) ** 2
    ratios = []
    for h in (0.0125, 0.00625):
        th = om * h
        N = 400
        s = O.Solver(p)
        s.set_state(psi, 0.0, h)
        s.step(N)
        decay = 1 - abs(np.vdot(pw, s.state()[0, 0]))
        decay -= 3 * th ** 6 / 144  # the 3 order-4 series start steps: |T4(i th)| = 1 - th^6/144
        ratios.append(decay / (N * th ** 6))
    r0 = 2 * ratios[1] - ratios[0]
    expect = -float(G["final"][1]) / 1.5
    assert r0 == pytest.approx(expect, rel=0.02), (ratios, r0, expect)
