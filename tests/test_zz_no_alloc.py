"""lise_rhs_noalloc: the right-hand side for callers that cannot allocate device
memory (a framework allocator owns the free memory, or cudaMalloc's implicit
synchronisation is not allowed where they run).  It is called here through the
C ABI on caller-owned device buffers, twice in a row with different inputs, and
each output is checked against the context-based lise_rhs entry point within
the single-right-hand-side tolerance the parity tests use (1e-12 relative).

The file name sorts last so that a run stopping at the first failure has run
every other test before this one.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2009_00745_b300 import lise as L

from .helpers import random_state, rel

pytestmark = pytest.mark.gpu

TOL_RHS = 1e-12


def _noalloc(p, psi_dev, t, out_dev):
    return L.load().lise_rhs_noalloc(C.byref(p), psi_dev.data_ptr(), float(t), out_dev.data_ptr())


@pytest.mark.parametrize("N,n_qp,precision,tol", [(16, 24, "fp64", TOL_RHS), (16, 24, "mixed", TOL_RHS),
                                                  (32, 24, "fp64", TOL_RHS), (48, 4, "fp64", TOL_RHS)])
def test_noalloc_matches_context_rhs_twice(N, n_qp, precision, tol):
    # (32^3 and 48^3 FP64 run the tensor-memory planes kernels with their core-matrix D2 tables)
    import torch
    from paper_2009_00745_b300 import build
    build.build()
    kw = dict(a=0.9, alpha=1.2, beta=-0.5, mu=0.35, g=0.8, drive_A=0.02, drive_Omega=0.3)
    vs = np.random.default_rng(5).uniform(-0.5, 0.5, (N, N, N))
    psis = [random_state(N, n_qp, seed=11), random_state(N, n_qp, seed=12, kmax=5)]
    times = [0.3, 1.7]
    # reference: the context-based entry point
    refs = []
    with L.Context(N, n_qp, v_static=vs, precision=precision, **kw) as ctx:
        for psi, t in zip(psis, times):
            refs.append(ctx.rhs(psi, t))
    p, keep = L._params(N, n_qp, kw["a"], kw["alpha"], kw["beta"], kw["mu"], kw["g"], vs, kw["drive_A"],
                        kw["drive_Omega"], precision, 0, 0, None)
    out = torch.empty((n_qp, 2, N, N, N), dtype=torch.complex128, device="cuda:0")
    xs = [torch.from_numpy(psi).to("cuda:0") for psi in psis]
    for k, (x, t, ref) in enumerate(zip(xs, times, refs)):
        out.fill_(float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(0)[0]
        rc = _noalloc(p, x, t, out)
        free1 = torch.cuda.mem_get_info(0)[0]
        assert rc == L.OK, L.strerror(rc)
        if k > 0:
            # after the first call (module loading, the symbol lookup) a call allocates nothing
            assert free1 == free0
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert rel(got, ref) < tol


def test_noalloc_rejects_oversized_problem():
    import torch
    N, n_qp = 32, 512  # 32 * 512 * 32^3 bytes of kinetic scratch alone: 512 MiB > 64 MiB
    p, _ = L._params(N, n_qp, 1.0, 1.0, 0.0, 0.0, 0.0, None, 0.0, 0.0, "fp64", 0, 0, None)
    x = torch.zeros(1, dtype=torch.complex128, device="cuda:0")
    assert _noalloc(p, x, 0.0, x) == L.ENOMEM


def test_noalloc_phase_removal_matches_context():
    import torch
    N, n_qp = 12, 10
    kw = dict(a=1.0, alpha=1.0, beta=-0.5, mu=0.3, g=0.9)
    psi = random_state(N, n_qp, seed=31, kmax=4)
    with L.Context(N, n_qp, remove_phase=True, **kw) as ctx:
        ref = ctx.rhs(psi, 0.7)
    p, keep = L._params(N, n_qp, kw["a"], kw["alpha"], kw["beta"], kw["mu"], kw["g"], None, 0.0, 0.0, "fp64",
                        0, 0, None, True)
    x = torch.from_numpy(psi).to("cuda:0")
    out = torch.empty_like(x)
    for _ in range(2):
        out.fill_(float("nan"))
        assert _noalloc(p, x, 0.7, out) == L.OK
        assert rel(out.cpu().numpy(), ref) < TOL_RHS


def test_noalloc_rejects_non_finite_parameters():
    # the same parameter checks as lise_create: a NaN coefficient never reaches a kernel
    import torch
    x = torch.zeros(1, dtype=torch.complex128, device="cuda:0")
    for field in ("alpha", "beta", "mu", "g", "drive_A", "drive_Omega", "pair_alpha"):
        p, _ = L._params(8, 2, 1.0, 1.0, -0.5, 0.1, 0.5, None, 0.01, 0.3, "fp64", 0, 0, None)
        setattr(p, field, float("nan"))
        assert _noalloc(p, x, 0.0, x) == L.EINVAL, field
