"""Seeded synthetic inputs for the two-component TDSLDA step.

This module only builds inputs (initial quasiparticle states, static external
potentials and the physical parameters of the named workloads).  It contains
none of the time-stepping arithmetic, and both the CUDA library and the CPU
oracle consume what it produces.  Numpy only.

Initial states are homogeneous BCS plane-wave quasiparticles, the positive
branch of the 2x2 Bogoliubov-de Gennes problem of Eq. hfb for a plane wave
(arXiv:2009.00745, Sec. "Nuclear DFT and SLDA"):

    u_k(r) = U_k e^{i k.r} / sqrt(Nxyz a^3),  v_k(r) = V_k e^{i k.r} / sqrt(Nxyz a^3),
    U_k = sqrt((1 + xi_k/E_k)/2),  V_k = sqrt((1 - xi_k/E_k)/2),
    E_k = sqrt(xi_k^2 + Delta0^2),  xi_k = (alpha/2) k^2 - mu0,

normalised as sum_r a^3 (|u|^2 + |v|^2) = 1 (the DVR orthonormality of
Sec. "Discretization").  The states are the n_qp lowest |k| on the lattice's
momentum grid, ties broken by the signed mode numbers (n_x, n_y, n_z) in
ascending order, each n in [-N/2, N/2).  mu0 = (alpha/2) k2_max / 2 with k2_max
the largest included k^2.

Gauge "noise" follows the boost/gauge transformation of Eq. kick with
chi(r) = (eps/2) xi(r), xi uniform in (-1, 1) drawn from SplitMix64 in site
order (x fastest); this puts the phase eps*xi(r) on nu and hence on Delta.
"""
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_MASK64 = (1 << 64) - 1


def splitmix64_uniform(seed: int, count: int) -> np.ndarray:
    """count doubles uniform in [-1, 1) from SplitMix64 (Steele, Lea, Flood 2014).

    Each output is (z >> 11) * 2^-53 mapped to [-1, 1), where z is the
    SplitMix64 output for the state seed + (i+1) * 0x9E3779B97F4A7C15.
    """
    with np.errstate(over="ignore"):
        i = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed & _MASK64) + i * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    u01 = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u01 - 1.0


def k_of_mode(n: int, N: int, a: float) -> float:
    """k for signed mode number n in [-N/2, N/2) (Sec. "Discretization")."""
    return 2.0 * np.pi * n / (N * a)


def lowest_modes(nx: int, ny: int, nz: int, a: float, n_qp: int) -> np.ndarray:
    """The n_qp lowest-|k| signed mode triples (mx, my, mz), sorted by
    (|k|^2, mx, my, mz)."""
    rx = np.arange(-(nx // 2), nx - nx // 2)
    ry = np.arange(-(ny // 2), ny - ny // 2)
    rz = np.arange(-(nz // 2), nz - nz // 2)
    MX, MY, MZ = np.meshgrid(rx, ry, rz, indexing="ij")
    MX, MY, MZ = MX.ravel(), MY.ravel(), MZ.ravel()
    kx = 2 * np.pi * MX / (nx * a)
    ky = 2 * np.pi * MY / (ny * a)
    kz = 2 * np.pi * MZ / (nz * a)
    k2 = kx * kx + ky * ky + kz * kz
    if nx == ny == nz:
        key_k2 = (MX * MX + MY * MY + MZ * MZ).astype(np.float64)  # exact ties on cubic lattices
    else:
        key_k2 = k2
    order = np.lexsort((MZ, MY, MX, key_k2))
    if n_qp > order.size:
        raise ValueError("n_qp exceeds the number of lattice modes")
    sel = order[:n_qp]
    return np.stack([MX[sel], MY[sel], MZ[sel]], axis=1)


def plane_wave(m, nx, ny, nz) -> np.ndarray:
    """exp(i k.r) on the lattice, (nz, ny, nx), exact phases via integer mods."""
    mx, my, mz = (int(v) for v in m)
    px = np.exp(2j * np.pi * ((mx * np.arange(nx)) % nx) / nx)
    py = np.exp(2j * np.pi * ((my * np.arange(ny)) % ny) / ny)
    pz = np.exp(2j * np.pi * ((mz * np.arange(nz)) % nz) / nz)
    return pz[:, None, None] * py[None, :, None] * px[None, None, :]


@dataclass
class Workload:
    """A named synthetic workload: parameters, initial state and step plan."""
    name: str
    nx: int
    ny: int
    nz: int
    a: float
    n_qp: int
    alpha: float
    beta: float
    mu: float
    g: float
    dt: float
    steps: int
    precision: str  # "fp64" or "mixed"
    v_static: Optional[np.ndarray] = None
    drive_A: float = 0.0
    drive_Omega: float = 0.0
    delta0: float = 0.5
    mu0: float = 0.0
    noise_eps: float = 0.0
    noise_seed: int = 42
    vortex: bool = False
    modes: Optional[np.ndarray] = field(default=None, repr=False)
    amps: Optional[np.ndarray] = field(default=None, repr=False)

    @property
    def nxyz(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def shape(self):
        return (self.n_qp, 2, self.nz, self.ny, self.nx)

    def qp_site_steps(self, steps: Optional[int] = None) -> float:
        return float(self.n_qp) * self.nxyz * (self.steps if steps is None else steps)

    def initial_state(self, q0: int = 0, q1: Optional[int] = None, out=None) -> np.ndarray:
        """States q0..q1-1 of the initial condition, shape (q1-q0, 2, nz, ny, nx)."""
        q1 = self.n_qp if q1 is None else q1
        nx, ny, nz = self.nx, self.ny, self.nz
        norm = 1.0 / np.sqrt(self.nxyz * self.a ** 3)
        psi = out if out is not None else np.empty((q1 - q0, 2, nz, ny, nx), dtype=np.complex128)
        gauge_u = np.ones((nz, ny, nx), dtype=np.complex128)
        gauge_v = np.ones((nz, ny, nx), dtype=np.complex128)
        if self.noise_eps:
            xi = splitmix64_uniform(self.noise_seed, self.nxyz).reshape(nz, ny, nx)
            chi = 0.5 * self.noise_eps * xi
            gauge_u = np.exp(1j * chi)
            gauge_v = np.exp(-1j * chi)
        if self.vortex:
            xc = (np.arange(nx) - nx // 2) * self.a
            yc = (np.arange(ny) - ny // 2) * self.a
            phi = np.arctan2(yc[:, None], xc[None, :])
            gauge_u = gauge_u * np.exp(1j * phi)[None, :, :]
        for j, q in enumerate(range(q0, q1)):
            pw = plane_wave(self.modes[q], nx, ny, nz) * norm
            U, V = self.amps[q]
            psi[j, 0] = U * pw * gauge_u
            psi[j, 1] = V * pw * gauge_v
        return psi


def _bcs(w: Workload) -> Workload:
    """Fill modes, BCS amplitudes, mu0 and the runtime mu (c.f. module doc)."""
    w.modes = lowest_modes(w.nx, w.ny, w.nz, w.a, w.n_qp)
    k2 = np.array([k_of_mode(m[0], w.nx, w.a) ** 2 + k_of_mode(m[1], w.ny, w.a) ** 2 +
                   k_of_mode(m[2], w.nz, w.a) ** 2 for m in w.modes])
    w.mu0 = 0.5 * w.alpha * k2.max() / 2.0
    xi = 0.5 * w.alpha * k2 - w.mu0
    E = np.sqrt(xi * xi + w.delta0 ** 2)
    U = np.sqrt(0.5 * (1.0 + xi / E))
    V = np.sqrt(0.5 * (1.0 - xi / E))
    w.amps = np.stack([U, V], axis=1)
    # Parameter choice (a gauge: mu only rotates u and v by opposite phases):
    # mu = mu0 + beta (3 pi^2 n0)^(2/3) / 2 with n0 the density of the
    # plane-wave state, so that the t = 0 diagonal of h equals xi_k exactly.
    n0 = 2.0 * np.sum(V * V) / (w.nxyz * w.a ** 3)
    w.mu = w.mu0 + 0.5 * w.beta * (3.0 * np.pi ** 2 * n0) ** (2.0 / 3.0)
    return w


def ufg_plane_waves(n: int, n_qp: int, *, steps=20, dt=0.005, noise_eps=1e-3, seed=42,
                    alpha=1.0, beta=-0.5, g=1.0, delta0=0.5, precision="fp64",
                    name=None) -> Workload:
    """Homogeneous unitary-Fermi-gas BCS plane waves on n^3 with gauge noise."""
    w = Workload(name or f"ufg{n}_{n_qp}", n, n, n, 1.0, n_qp, alpha, beta, 0.0, g, dt, steps,
                 precision, delta0=delta0, noise_eps=noise_eps, noise_seed=seed)
    return _bcs(w)


def harmonic_trap(n: int, omega: float, a: float = 1.0) -> np.ndarray:
    """V = omega^2 r^2 / 2 with r measured from the box centre ((i - n/2) a)."""
    c = (np.arange(n) - n // 2) * a
    r2 = c[None, None, :] ** 2 + c[None, :, None] ** 2 + c[:, None, None] ** 2
    return 0.5 * omega * omega * r2


def trap_vortex(n: int = 32, n_qp: int = 2048, *, steps=1000, dt=0.005, omega=0.1,
                alpha=1.0, beta=-0.5, g=1.0, delta0=0.5, precision="fp64", name=None) -> Workload:
    """Plane-wave BCS states in a harmonic trap with a straight vortex phase
    e^{i phi(x, y)} on every u (so nu and Delta wind once around z)."""
    w = Workload(name or f"trap{n}_vortex_{n_qp}", n, n, n, 1.0, n_qp, alpha, beta, 0.0, g, dt,
                 steps, precision, v_static=harmonic_trap(n, omega), delta0=delta0, vortex=True)
    return _bcs(w)


def driven(n: int = 48, n_qp: int = 4096, *, steps=1000, dt=0.005, A=0.01, Omega=0.3,
           noise_eps=1e-3, seed=42, alpha=1.0, beta=-0.5, g=1.0, delta0=0.5,
           precision="mixed", name=None) -> Workload:
    """Plane-wave BCS states (with gauge noise) under V_ext = A sin(Omega t) z."""
    w = Workload(name or f"drive{n}_{n_qp}", n, n, n, 1.0, n_qp, alpha, beta, 0.0, g, dt, steps,
                 precision, drive_A=A, drive_Omega=Omega, delta0=delta0, noise_eps=noise_eps,
                 noise_seed=seed)
    return _bcs(w)


def named(name: str, n_qp: Optional[int] = None) -> Workload:
    """The standard workloads by name (n_qp overrides the state count; the name
    then carries the count as a suffix).

    ufg16_fp64            16^3 x 256 states, dt 0.005, 20 steps, FP64
    trap32_vortex_fp64    32^3 x 2048 states, trap omega 0.1 + vortex, 1000 steps, FP64
    drive48_mixed         48^3 x 4096 states, drive A 0.01 Omega 0.3, 1000 steps, mixed
    drive48_fp64_small    48^3 x 256 states, the drive workload reduced for the oracle, 20 steps
    """
    table = {
        "ufg16_fp64": lambda q: ufg_plane_waves(16, q or 256, steps=20, name=name),
        "trap32_vortex_fp64": lambda q: trap_vortex(32, q or 2048, steps=1000, name=name),
        "drive48_mixed": lambda q: driven(48, q or 4096, steps=1000, precision="mixed", name=name),
        "drive48_fp64_small": lambda q: driven(48, q or 256, steps=20, precision="fp64", name=name),
    }
    if name not in table:
        raise KeyError(name)
    w = table[name](n_qp)
    if n_qp is not None:
        w.name = f"{name}:{n_qp}"
    return w
