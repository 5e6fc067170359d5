"""ctypes wrapper of the FP64 CPU oracle (oracle/lise_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check and
by the benchmark's CPU-baseline leg, never by the library itself.  The oracle
follows arXiv:2009.00745 (Sec. "Discretization", Eq. tdslda, Eqs. rho_t/nu_t,
Eq. pairingfield, Sec. TDSLDA "Time evolution", Eqs. p, m, c, y); see
lise_oracle.h for the readings it takes where the paper is silent.

State arrays are complex128 with shape (n_qp, 2, nz, ny, nx): component 0 is u,
component 1 is v.  Densities/potentials have shape (nz, ny, nx).
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.POINTER
        d, i, vp = C.c_double, C.c_int, C.c_void_p
        L.or_dft1d.argtypes = [vp, vp, i, i]
        L.or_fft3d.argtypes = [vp, i, i, i, i]
        L.or_kgrid.argtypes = [i, i, d]
        L.or_kgrid.restype = d
        L.or_kinetic.argtypes = [vp, vp, vp]
        L.or_densities.argtypes = [vp, vp, vp, vp]
        L.or_potentials.argtypes = [vp, vp, vp, d, vp, vp]
        L.or_apply_h.argtypes = [vp, vp, vp, vp, vp]
        L.or_rhs.argtypes = [vp, vp, d, vp]
        L.or_kick.argtypes = [vp, vp, vp]
        L.or_gradient.argtypes = [vp, vp, i, vp]
        L.or_currents.argtypes = [vp, vp, vp]
        L.or_solver_kick.argtypes = [vp, vp]
        L.or_solver_kick.restype = i
        L.or_create.argtypes = [vp]
        L.or_create.restype = vp
        L.or_destroy.argtypes = [vp]
        L.or_set_state.argtypes = [vp, vp, d, d]
        L.or_set_state.restype = i
        L.or_step.argtypes = [vp, i]
        L.or_step.restype = i
        L.or_set_history.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, d, d]
        L.or_set_history.restype = i
        L.or_get_state.argtypes = [vp, vp]
        L.or_time.argtypes = [vp]
        L.or_time.restype = d
        L.or_get_densities.argtypes = [vp, vp, vp]
        L.or_energy.argtypes = [vp, P(d), P(d)]
        L.or_energy_of.argtypes = [vp, vp, d, P(d), P(d)]
        L.or_series_step.argtypes = [vp, vp, d, d, vp]
        L.or_num_threads.restype = i
        L.or_abm_predictor.argtypes = [C.c_long, d, vp, vp, vp, vp, vp, vp, vp]
        L.or_abm_modifier.argtypes = [C.c_long, vp, vp, vp]
        L.or_abm_corrector.argtypes = [C.c_long, d, vp, vp, vp, vp, vp, vp, vp]
        L.or_abm_final.argtypes = [C.c_long, vp, vp, vp, vp]
        L.or_eta.argtypes = [vp, vp, vp, vp]
        L.or_geff.argtypes = [vp, d, d, P(d), P(d)]
        _lib = L
    return _lib


class _Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("a", C.c_double),
                ("n_qp", C.c_int), ("alpha", C.c_double), ("beta", C.c_double),
                ("mu", C.c_double), ("g", C.c_double), ("v_static", C.c_void_p),
                ("drive_A", C.c_double), ("drive_Omega", C.c_double), ("remove_phase", C.c_int),
                ("pair_alpha", C.c_double), ("pair_n0", C.c_double), ("pair_lattice", C.c_int),
                ("renormalize", C.c_int), ("pair_ec", C.c_double)]


class Params:
    """Physical and lattice parameters (ħ = m = 1)."""

    def __init__(self, nx, ny, nz, a=1.0, n_qp=1, alpha=1.0, beta=0.0, mu=0.0, g=0.0,
                 v_static=None, drive_A=0.0, drive_Omega=0.0, remove_phase=False, pair_alpha=0.0,
                 pair_n0=1.0, pair_lattice=False, renormalize=False, pair_ec=0.0):
        self.nx, self.ny, self.nz, self.a, self.n_qp = int(nx), int(ny), int(nz), float(a), int(n_qp)
        self.alpha, self.beta, self.mu, self.g = float(alpha), float(beta), float(mu), float(g)
        self.v_static = None if v_static is None else np.ascontiguousarray(v_static, dtype=np.float64).reshape(nz, ny, nx)
        self.drive_A, self.drive_Omega = float(drive_A), float(drive_Omega)
        self.remove_phase = bool(remove_phase)
        self.pair_alpha, self.pair_n0, self.pair_lattice = float(pair_alpha), float(pair_n0), bool(pair_lattice)
        self.renormalize = bool(renormalize)
        self.pair_ec = float(pair_ec)

    def with_(self, **kw):
        d = dict(nx=self.nx, ny=self.ny, nz=self.nz, a=self.a, n_qp=self.n_qp, alpha=self.alpha,
                 beta=self.beta, mu=self.mu, g=self.g, v_static=self.v_static,
                 drive_A=self.drive_A, drive_Omega=self.drive_Omega, remove_phase=self.remove_phase,
                 pair_alpha=self.pair_alpha, pair_n0=self.pair_n0, pair_lattice=self.pair_lattice,
                 renormalize=self.renormalize, pair_ec=self.pair_ec)
        d.update(kw)
        return Params(**d)

    def _c(self):
        s = _Params(self.nx, self.ny, self.nz, self.a, self.n_qp, self.alpha, self.beta, self.mu,
                    self.g, None if self.v_static is None else self.v_static.ctypes.data,
                    self.drive_A, self.drive_Omega, int(self.remove_phase), self.pair_alpha,
                    self.pair_n0, int(self.pair_lattice), int(self.renormalize), self.pair_ec)
        return s

    @property
    def shape(self):
        return (self.n_qp, 2, self.nz, self.ny, self.nx)

    @property
    def grid(self):
        return (self.nz, self.ny, self.nx)


def _c128(x, shape=None):
    a = np.ascontiguousarray(x, dtype=np.complex128)
    if shape is not None:
        a = a.reshape(shape)
    return a


def dft1d(x, sign=-1):
    x = _c128(x)
    out = np.empty_like(x)
    lib().or_dft1d(x.ctypes.data, out.ctypes.data, x.size, sign)
    return out


def fft3d(vol, sign=-1):
    v = _c128(vol).copy()
    nz, ny, nx = v.shape
    lib().or_fft3d(v.ctypes.data, nx, ny, nz, sign)
    return v


def kgrid(idx, n, a):
    return lib().or_kgrid(idx, n, a)


def kinetic(p: Params, f):
    f = _c128(f, p.grid)
    out = np.empty_like(f)
    ps = p._c()
    lib().or_kinetic(C.byref(ps), f.ctypes.data, out.ctypes.data)
    return out


def densities(p: Params, psi):
    psi = _c128(psi, p.shape)
    n = np.empty(p.grid)
    nu = np.empty(p.grid, dtype=np.complex128)
    ps = p._c()
    lib().or_densities(C.byref(ps), psi.ctypes.data, n.ctypes.data, nu.ctypes.data)
    return n, nu


def potentials(p: Params, n, nu, t):
    n = np.ascontiguousarray(n, dtype=np.float64).reshape(p.grid)
    nu = _c128(nu, p.grid)
    W = np.empty(p.grid)
    D = np.empty(p.grid, dtype=np.complex128)
    ps = p._c()
    lib().or_potentials(C.byref(ps), n.ctypes.data, nu.ctypes.data, float(t), W.ctypes.data, D.ctypes.data)
    return W, D


def apply_h(p: Params, W, D, psi):
    W = np.ascontiguousarray(W, dtype=np.float64).reshape(p.grid)
    D = _c128(D, p.grid)
    psi = _c128(psi, p.shape)
    out = np.empty_like(psi)
    ps = p._c()
    lib().or_apply_h(C.byref(ps), W.ctypes.data, D.ctypes.data, psi.ctypes.data, out.ctypes.data)
    return out


def rhs(p: Params, psi, t):
    psi = _c128(psi, p.shape)
    out = np.empty_like(psi)
    ps = p._c()
    lib().or_rhs(C.byref(ps), psi.ctypes.data, float(t), out.ctypes.data)
    return out


def series_step(p: Params, psi, t, dt):
    psi = _c128(psi, p.shape)
    out = np.empty_like(psi)
    ps = p._c()
    lib().or_series_step(C.byref(ps), psi.ctypes.data, float(t), float(dt), out.ctypes.data)
    return out


def eta(p: Params, psi, hpsi):
    """eta_k = <psi_k|H psi_k> (real part), one value per state (Eq. sp_en)."""
    psi = _c128(psi, p.shape)
    hpsi = _c128(hpsi, p.shape)
    out = np.empty(p.n_qp)
    ps = p._c()
    lib().or_eta(C.byref(ps), psi.ctypes.data, hpsi.ctypes.data, out.ctypes.data)
    return out


def gradient(p: Params, f, axis):
    """F^-1[(ik) F f] along axis 0 = x, 1 = y, 2 = z, Nyquist coefficient dropped."""
    f = _c128(f, p.grid)
    out = np.empty(p.grid, dtype=np.complex128)
    ps = p._c()
    lib().or_gradient(C.byref(ps), f.ctypes.data, int(axis), out.ctypes.data)
    return out


def currents(p: Params, psi):
    """Current density of Eq. j (spin factor 2): j[3][z][y][x], components x, y, z."""
    psi = _c128(psi, p.shape)
    out = np.empty((3,) + p.grid)
    ps = p._c()
    lib().or_currents(C.byref(ps), psi.ctypes.data, out.ctypes.data)
    return out


def kick(p: Params, psi, chi):
    """Eq. kick: u -> exp(i chi) u, v -> exp(-i chi) v (returns a new array)."""
    out = _c128(psi, p.shape).copy()
    chi = np.ascontiguousarray(chi, dtype=np.float64).reshape(p.grid)
    ps = p._c()
    lib().or_kick(C.byref(ps), out.ctypes.data, chi.ctypes.data)
    return out


def geff(p: Params, n, u_loc=0.0):
    """(g_eff, d g_eff / dn) at density n and local potential u_loc = U(n) + V_ext."""
    g, dg = C.c_double(), C.c_double()
    ps = p._c()
    lib().or_geff(C.byref(ps), float(n), float(u_loc), C.byref(g), C.byref(dg))
    return g.value, dg.value


def energy_of(p: Params, psi, t):
    psi = _c128(psi, p.shape)
    E, N = C.c_double(), C.c_double()
    ps = p._c()
    lib().or_energy_of(C.byref(ps), psi.ctypes.data, float(t), C.byref(E), C.byref(N))
    return E.value, N.value


def abm_predictor(h, yn, ynm1, d0, d1, d2, d3):
    """Eq. p elementwise (the integrator's own routine)."""
    a = [_c128(x).ravel() for x in (yn, ynm1, d0, d1, d2, d3)]
    out = np.empty_like(a[0])
    lib().or_abm_predictor(a[0].size, float(h), *[x.ctypes.data for x in a], out.ctypes.data)
    return out


def abm_modifier(p, pc):
    """Eq. m elementwise."""
    p, pc = _c128(p).ravel(), _c128(pc).ravel()
    out = np.empty_like(p)
    lib().or_abm_modifier(p.size, p.ctypes.data, pc.ctypes.data, out.ctypes.data)
    return out


def abm_corrector(h, yn, ynm1, mp, d0, d1, d2):
    """Eq. c elementwise."""
    a = [_c128(x).ravel() for x in (yn, ynm1, mp, d0, d1, d2)]
    out = np.empty_like(a[0])
    lib().or_abm_corrector(a[0].size, float(h), *[x.ctypes.data for x in a], out.ctypes.data)
    return out


def abm_final(p, c):
    """Eq. y elementwise; returns (y_{n+1}, p_{n+1} - c_{n+1})."""
    p, c = _c128(p).ravel(), _c128(c).ravel()
    y = np.empty_like(p)
    pc = np.empty_like(p)
    lib().or_abm_final(p.size, p.ctypes.data, c.ctypes.data, y.ctypes.data, pc.ctypes.data)
    return y, pc


def num_threads():
    return lib().or_num_threads()


class Solver:
    """Series-expansion start + ABM integrator of the oracle."""

    def __init__(self, p: Params):
        self.p = p
        self._ps = p._c()  # keeps v_static alive via p
        self._h = lib().or_create(C.byref(self._ps))

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_destroy(self._h)
            self._h = None

    def set_state(self, psi, t0, dt):
        psi = _c128(psi, self.p.shape)
        rc = lib().or_set_state(self._h, psi.ctypes.data, float(t0), float(dt))
        if rc:
            raise ValueError("oracle set_state failed")

    def set_history(self, yn, ynm1, d, t, dt, pc=None):
        """Load an ABM history directly (no series start): y_n, y_{n-1}, the four
        derivatives d = [y'_n, y'_{n-1}, y'_{n-2}, y'_{n-3}], p_n - c_n (None: zero),
        at time t with step dt."""
        arrs = [_c128(x, self.p.shape) for x in [yn, ynm1] + list(d)]
        pcp = None if pc is None else _c128(pc, self.p.shape)
        rc = lib().or_set_history(self._h, *[a.ctypes.data for a in arrs],
                                  None if pcp is None else pcp.ctypes.data, float(t), float(dt))
        if rc:
            raise ValueError("oracle set_history failed")

    def kick(self, chi):
        """Eq. kick on the current state, then a new series start at the current time."""
        chi = np.ascontiguousarray(chi, dtype=np.float64).reshape(self.p.grid)
        if lib().or_solver_kick(self._h, chi.ctypes.data):
            raise RuntimeError("oracle kick before set_state")

    def step(self, n):
        rc = lib().or_step(self._h, int(n))
        if rc:
            raise RuntimeError("oracle step before set_state")

    def state(self):
        out = np.empty(self.p.shape, dtype=np.complex128)
        lib().or_get_state(self._h, out.ctypes.data)
        return out

    @property
    def t(self):
        return lib().or_time(self._h)

    def densities(self):
        n = np.empty(self.p.grid)
        nu = np.empty(self.p.grid, dtype=np.complex128)
        lib().or_get_densities(self._h, n.ctypes.data, nu.ctypes.data)
        return n, nu

    def energy(self):
        E, N = C.c_double(), C.c_double()
        lib().or_energy(self._h, C.byref(E), C.byref(N))
        return E.value, N.value
