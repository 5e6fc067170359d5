"""The C ABI library loads and exports every entry point include/lise.h declares;
host-side argument checks (no GPU needed, no device call made)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2009_00745_b300 import build as B
from paper_2009_00745_b300 import lise as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lise.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lise_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    # the binding covers the same set
    assert set(names) == set(L.SIGNATURES)


def test_strerror(lib):
    assert L.strerror(L.OK) == "ok"
    assert "budget" in L.strerror(L.ENOMEM)
    assert L.strerror(999) == "unknown status"


def test_footprint_model():
    f16 = L.footprint_bytes(16, 256)
    f32 = L.footprint_bytes(32, 2048)
    assert f16 > 11 * 16 * 256 * 2 * 16 ** 3   # at least the 10 history arrays + scratch
    # state arrays dominate: 11 complex128 copies of 2048 x 2 x 32^3 (10 history + scratch)
    assert abs(f32 - 11 * 16 * 2048 * 2 * 32 ** 3) / f32 < 0.02
    fm = L.footprint_bytes(48, 4096, precision="mixed")
    # mixed: y_n, y_{n-1}, Q in complex128; the y' ring, m, R, p - c and T_xy in complex64
    assert abs(fm - (3 * 16 + 8 * 8) * 4096 * 2 * 48 ** 3) / fm < 0.02
    fs = L.footprint_bytes(48, 4096, precision="mixed_strict")
    # strict split: R and p - c in complex128 as well
    assert abs(fs - (5 * 16 + 6 * 8) * 4096 * 2 * 48 ** 3) / fs < 0.02
    assert L.footprint_bytes(30, 8) == 0  # unsupported lattice


def _create(**kw):
    base = dict(N=16, n_qp=8)
    base.update(kw)
    N = base.pop("N")
    n_qp = base.pop("n_qp")
    return L.Context(N, n_qp, **base)


@pytest.mark.parametrize("kw", [dict(N=30), dict(N=16, n_qp=0), dict(N=16, a=0.0), dict(N=16, precision=7),
                                dict(N=16, beta=float("nan"))])
def test_invalid_parameters(kw):
    with pytest.raises(L.LiseError) as e:
        _create(**kw)
    assert e.value.status == L.EINVAL


def test_non_cubic_rejected(lib):
    p = L._Params(16, 16, 32, 1.0, 4, 1.0, 0.0, 0.0, 0.0, None, 0.0, 0.0, 0, 0, 0, None)
    h = C.c_void_p()
    assert lib.lise_create(C.byref(p), C.byref(h)) == L.EINVAL
    assert lib.lise_footprint_bytes(C.byref(p)) == 0


def test_budget_rejected_before_any_allocation():
    need = L.footprint_bytes(32, 2048)
    with pytest.raises(L.LiseError) as e:
        _create(N=32, n_qp=2048, hbm_budget_bytes=need - 1)
    assert e.value.status == L.ENOMEM


def test_null_arguments(lib):
    assert lib.lise_create(None, None) == L.EINVAL
    assert lib.lise_step(None, 1, 0.1) == L.EINVAL
    assert lib.lise_sync(None) == L.EINVAL
    assert lib.lise_set_wait_limit(None, 0) == L.EINVAL
    lib.lise_destroy(None)


@pytest.mark.parametrize("field", ["alpha", "beta", "mu", "g", "drive_A", "drive_Omega", "dx"])
def test_noalloc_validates_parameters_before_any_device_call(lib, field):
    # lise_rhs_noalloc applies lise_create's checks first: a non-finite parameter is
    # rejected without touching the (here absent) device; the buffer addresses are never used
    p, _ = L._params(16, 4, 1.0, 1.0, -0.5, 0.2, 0.7, None, 0.01, 0.3, "fp64", 0, 0, None)
    setattr(p, field, float("nan"))
    fake = C.c_void_p(4096)
    assert lib.lise_rhs_noalloc(C.byref(p), fake, 0.0, fake) == L.EINVAL
    p.dx = 1.0
    p.alpha = p.beta = p.mu = p.g = p.drive_A = p.drive_Omega = 0.0
    p.pair_alpha, p.pair_n0 = 0.5, 0.0   # Eq. g0 needs n0 > 0
    assert lib.lise_rhs_noalloc(C.byref(p), fake, 0.0, fake) == L.EINVAL


@pytest.mark.parametrize("ec,lattice,alpha,ok", [
    (0.0, 0, 1.0, True), (2.0, 0, 1.0, True), (np.pi ** 2 / 2, 0, 1.0, True),
    (np.pi ** 2 / 2 * 1.0001, 0, 1.0, False),   # above the natural cutoff of one axis
    (2.0, 1, 1.0, False),                       # not with the lattice form of Eq. geff_3D
    (-0.1, 0, 1.0, False), (float("nan"), 0, 1.0, False), (float("inf"), 0, 1.0, False),
    (1.0, 0, 0.0, False)])
def test_spherical_cutoff_parameters(lib, ec, lattice, alpha, ok):
    # Eq. geff: 0 < E_c <= alpha pi^2 / (2 dx^2); lise_footprint_bytes is 0 for invalid parameters
    p, _ = L._params(16, 4, 1.0, alpha, -0.5, 0.2, -0.7, None, 0.0, 0.0, "fp64", 0, 0, None,
                     pair_lattice=bool(lattice), pair_ec=ec)
    assert (lib.lise_footprint_bytes(C.byref(p)) > 0) == ok
    if not ok:
        fake = C.c_void_p(4096)
        assert lib.lise_rhs_noalloc(C.byref(p), fake, 0.0, fake) == L.EINVAL


def test_pencil_batch_controls_host_only():
    # host-side table of the pencil autotuner: no device call
    assert L.pencil_batch(30) == 0                       # unsupported lattice
    assert L.pencil_batch(32, "fp64") in (2, 4)
    with pytest.raises(L.LiseError) as e:
        L.set_pencil_batch(32, "fp64", 3)                # no such variant
    assert e.value.status == L.EINVAL
    L.set_pencil_batch(16, "mixed", 4)
    assert L.pencil_batch(16, "mixed") == 4
    L.set_pencil_batch(16, "mixed", 0)                   # back to the default / next tuning
    assert L.pencil_batch(16, "mixed") in (2, 4)
    L.set_pencil_batch(32, "fp64", 1)                    # one state per batch: FP64 tensor-core kernel only
    assert L.pencil_batch(32, "fp64") == 1
    L.set_pencil_batch(32, "fp64", 0)
    with pytest.raises(L.LiseError) as e:
        L.set_pencil_batch(16, "mixed", 1)
    assert e.value.status == L.EINVAL
    with pytest.raises(L.LiseError) as e:
        L.set_pencil_batch(24, "fp64", 1)                # 24 % 16 != 0: FFT kernels
    assert e.value.status == L.EINVAL


def test_planes_per_block_controls_host_only():
    assert L.planes_per_block(32, "fp64") == 0          # tensor-core planes kernel
    assert L.planes_per_block(48, "mixed") in (1, 2, 4, 8, -1, -2, -4, -8)
    with pytest.raises(L.LiseError) as e:
        L.set_planes_per_block(32, "fp64", 2)           # no FFT planes kernel there
    assert e.value.status == L.EINVAL
    with pytest.raises(L.LiseError) as e:
        L.set_planes_per_block(64, "mixed", 8)          # 8 planes of 64^2 do not fit
    assert e.value.status == L.EINVAL
    L.set_planes_per_block(16, "mixed", 8)
    assert L.planes_per_block(16, "mixed") == 8
    L.set_planes_per_block(16, "mixed", -4)             # whole lines in registers
    assert L.planes_per_block(16, "mixed") == -4
    for N, prec, pb in ((64, "mixed", -8), (12, "fp64", -2), (16, "mixed", -3)):
        with pytest.raises(L.LiseError) as e:           # no register-line variant there
            L.set_planes_per_block(N, prec, pb)
        assert e.value.status == L.EINVAL
    L.set_planes_per_block(16, "mixed", 0)
