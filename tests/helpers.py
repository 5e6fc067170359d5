"""Shared test helpers: workload -> oracle parameters, error norms, GPU gate."""
import numpy as np

from oracle import oracle as O


def oracle_params(w, **kw):
    p = O.Params(w.nx, w.ny, w.nz, a=w.a, n_qp=w.n_qp, alpha=w.alpha, beta=w.beta, mu=w.mu,
                 g=w.g, v_static=w.v_static, drive_A=w.drive_A, drive_Omega=w.drive_Omega)
    return p.with_(**kw) if kw else p


def rel(a, b):
    """||a - b||_2 / ||b||_2 over the whole array."""
    return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def random_state(N, n_qp, seed, kmax=None):
    """Normalised random states; band-limited to |m| <= kmax per axis if kmax is given."""
    rng = np.random.default_rng(seed)
    shape = (n_qp, 2, N, N, N)
    psi = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    if kmax is not None:
        f = np.fft.fftn(psi, axes=(2, 3, 4))
        m = np.abs(np.fft.fftfreq(N, 1.0 / N))
        keep = (m[:, None, None] <= kmax) & (m[None, :, None] <= kmax) & (m[None, None, :] <= kmax)
        f *= keep
        psi = np.fft.ifftn(f, axes=(2, 3, 4))
    psi /= np.sqrt(np.sum(np.abs(psi) ** 2, axis=(1, 2, 3, 4), keepdims=True))
    return psi
