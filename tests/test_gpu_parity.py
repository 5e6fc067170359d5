"""GPU parity: the CUDA library through its C ABI against the FP64 CPU oracle.

FP64 path tolerance (after a whole run): ||x_gpu - x_oracle||_2 / ||x_oracle||_2
<= 1e-11 for psi, n and nu.  A single right-hand side is held to 1e-12.  The
mixed path (complex64 FFTs and H psi, FP64 history) is held to the bound its
arithmetic allows, derived in the individual tests.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2009_00745_b300 import lise as L
from paper_2009_00745_b300 import workloads as W

from .helpers import oracle_params, random_state, rel

pytestmark = pytest.mark.gpu

TOL_FP64_RUN = 1e-11
TOL_FP64_RHS = 1e-12
TOL_FP64_ELEM = 1e-10   # per element, relative to the largest element of the array


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2009_00745_b300 import build
    build.build()
    L.load()


# ------------------------------------------------------------ one RHS ----

@pytest.mark.parametrize("N,n_qp", [(8, 5), (12, 7), (16, 9), (20, 3), (24, 6), (32, 5), (40, 3), (48, 2),
                                    (64, 1)])
def test_rhs_all_lattices(N, n_qp):
    psi = random_state(N, n_qp, seed=N)
    kw = dict(a=0.8, alpha=1.3, beta=-0.5, mu=0.4, g=0.7)
    rng = np.random.default_rng(1)
    vs = rng.uniform(-1, 1, (N, N, N))
    with L.Context(N, n_qp, v_static=vs, drive_A=0.02, drive_Omega=0.3, **kw) as ctx:
        got = ctx.rhs(psi, 0.9)
    p = O.Params(N, N, N, n_qp=n_qp, v_static=vs, drive_A=0.02, drive_Omega=0.3, **kw)
    ref = O.rhs(p, psi, 0.9)
    assert rel(got, ref) < TOL_FP64_RHS


@pytest.mark.parametrize("N", [16, 32])
def test_rhs_wide_dynamic_range(N):
    # The FP64 kinetic operator on the tensor cores scales each (state, component,
    # re/im) group of a tile by its own binary exponent: every state and component
    # keeps FP64 accuracy relative to its own size, here across 12 decades and with
    # an identically zero component (its group has exponent field 0).
    n_qp = 6
    psi = random_state(N, n_qp, seed=11)
    scale = np.array([1.0, 1e-3, 1e-6, 1e-9, 1e-12, 1.0])
    psi *= scale[:, None, None, None, None]
    psi[1, 1] *= 1e-4          # v much smaller than u
    psi[5, 1] = 0.0            # v identically zero
    kw = dict(alpha=1.0, beta=-0.5, mu=0.3, g=0.8)
    with L.Context(N, n_qp, **kw) as ctx:
        got = ctx.rhs(psi, 0.0)
    ref = O.rhs(O.Params(N, N, N, n_qp=n_qp, **kw), psi, 0.0)
    for q in range(n_qp):
        for c in range(2):
            if not np.any(ref[q, c]):
                continue
            assert rel(got[q, c], ref[q, c]) < 1e-12, (q, c, rel(got[q, c], ref[q, c]))
    assert np.all(np.isfinite(got))


def test_rhs_mixed_precision_bound():
    N, n_qp = 24, 6
    psi = random_state(N, n_qp, seed=3, kmax=6)
    kw = dict(alpha=1.0, beta=-0.5, mu=0.3, g=1.0)
    with L.Context(N, n_qp, precision="mixed", **kw) as ctx:
        got = ctx.rhs(psi, 0.0)
    ref = O.rhs(O.Params(N, N, N, n_qp=n_qp, **kw), psi, 0.0)
    # FP32 transforms: a few units of 2^-24 times log2(N^3) butterflies
    err = rel(got, ref)
    assert err < 2e-6, err
    assert err > 1e-12  # it is really FP32 arithmetic


@pytest.mark.parametrize("N,n_qp", [(8, 5), (12, 7), (20, 3), (32, 3), (64, 1)])
def test_rhs_mixed_all_lattices(N, n_qp):
    # the FP32 compute precision on the other lattice families: z-pencil tiles 8 wide (8^3,
    # 32^3, 64^3) and 4 wide (12^3, 20^3), i.e. both widths of the staged batch boxes, and the
    # radix plans 2x4, 4x3, 4x5, 4x8, 8x8
    psi = random_state(N, n_qp, seed=N + 100, kmax=max(1, N // 4))
    kw = dict(a=0.9, alpha=1.0, beta=-0.5, mu=0.3, g=1.0)
    rng = np.random.default_rng(2)
    vs = rng.uniform(-1, 1, (N, N, N))
    with L.Context(N, n_qp, precision="mixed", v_static=vs, **kw) as ctx:
        got = ctx.rhs(psi, 0.0)
    ref = O.rhs(O.Params(N, N, N, n_qp=n_qp, v_static=vs, **kw), psi, 0.0)
    err = rel(got, ref)
    assert err < 2e-6, err
    assert err > 1e-12


# ------------------------------------------------------------ full runs ----

def run_gpu(w, steps, precision="fp64"):
    with L.Context.from_workload(w, precision=precision) as ctx:
        ctx.set_state(w.initial_state(), 0.0, w.dt)
        ctx.step(steps)
        psi = ctx.state()
        n, nu = ctx.densities()
        E, N = ctx.energy()
        t = ctx.t
    return psi, n, nu, E, N, t


def run_oracle(w, steps):
    s = O.Solver(oracle_params(w))
    s.set_state(w.initial_state(), 0.0, w.dt)
    s.step(steps)
    n, nu = s.densities()
    E, N = s.energy()
    return s.state(), n, nu, E, N, s.t


def maxabs_rel(a, b):
    """max |a - b| / max |b| over all elements: a local error (one tile, one boundary
    plane) that a whole-array norm would dilute shows here."""
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / np.max(np.abs(np.asarray(b))))


def check_run(w, steps):
    g = run_gpu(w, steps)
    o = run_oracle(w, steps)
    assert g[5] == pytest.approx(o[5], abs=1e-14)
    assert rel(g[0], o[0]) < TOL_FP64_RUN, "psi"
    assert rel(g[1], o[1]) < TOL_FP64_RUN, "n"
    assert rel(g[2], o[2]) < TOL_FP64_RUN, "nu"
    for k, name in ((0, "psi"), (1, "n"), (2, "nu")):
        assert maxabs_rel(g[k], o[k]) < TOL_FP64_ELEM, name
    assert g[3] == pytest.approx(o[3], rel=1e-11, abs=1e-11)
    assert g[4] == pytest.approx(o[4], rel=1e-12)
    return g, o


def test_ufg16_full_workload():
    # 16^3 lattice, 256 states, dt 0.005, 20 ABM steps, gauge noise seed 42
    w = W.named("ufg16_fp64")
    check_run(w, w.steps)


@pytest.mark.parametrize("N,n_qp,steps", [(8, 13, 12), (12, 9, 6), (20, 11, 5), (24, 37, 4), (40, 5, 3)])
def test_ragged_state_counts(N, n_qp, steps):
    w = W.ufg_plane_waves(N, n_qp, noise_eps=0.05, steps=steps)
    check_run(w, steps)


def test_trap_vortex_reduced():
    w = W.trap_vortex(32, 24, steps=8)
    check_run(w, w.steps)


def test_drive_reduced():
    w = W.driven(48, 6, steps=6, precision="fp64")
    check_run(w, w.steps)


def test_drive_48_cubed_256_states_20_steps():
    # the driven 48^3 workload reduced to 256 states (the oracle's full 4096-state history
    # would not fit a host), 20 ABM steps after the start, FP64
    w = W.named("drive48_fp64_small")
    assert (w.nx, w.n_qp, w.steps) == (48, 256, 20)
    check_run(w, w.steps)


@pytest.mark.parametrize("N,precision", [(16, "fp64"), (32, "fp64"), (24, "mixed")])
def test_drive_closed_form(N, precision):
    # alpha = beta = g = 0: every site rotates by exp(-i int (V_ext - mu) dt) with
    # V_ext = A sin(Omega t) z_c (Sec. "External boosts and external potentials"); the GPU
    # follows the oracle (whose drive and evaluation times are pinned on the CPU against
    # this closed form) and its error against the closed form has the drive's shape z_c
    n_qp, A, Om, mu, dt, steps = 6, 0.3, 2.0, 0.1, 0.01, 12
    psi0 = random_state(N, n_qp, seed=N + 7)
    kw = dict(alpha=0.0, beta=0.0, mu=mu, g=0.0, drive_A=A, drive_Omega=Om)
    with L.Context(N, n_qp, precision=precision, **kw) as ctx:
        ctx.set_state(psi0, 0.2, dt)
        ctx.step(steps)
        got, t = ctx.state(), ctx.t
    s = O.Solver(O.Params(N, N, N, n_qp=n_qp, **kw))
    s.set_state(psi0, 0.2, dt)
    s.step(steps)
    assert t == pytest.approx(s.t, abs=1e-14)
    tol = TOL_FP64_RUN if precision == "fp64" else 2e-6
    assert rel(got, s.state()) < tol
    zc = ((np.arange(N) - N // 2) * 1.0)[:, None, None] * np.ones((1, N, N))
    ph = -mu * (t - 0.2) + A * zc * (np.cos(Om * 0.2) - np.cos(Om * t)) / Om
    exact = psi0.copy()
    exact[:, 0] *= np.exp(-1j * ph)
    exact[:, 1] *= np.exp(1j * ph)
    err = np.angle(got[:, 0] / exact[:, 0])
    # the start's midpoint-rule remainders (cubic in dt, linear in z_c); nothing on z = N/2
    bound = 3 * dt ** 3 / 24 * A * Om ** 2 * (N // 2)
    assert np.max(np.abs(err)) < 1.2 * bound + (1e-5 if precision == "mixed" else 0.0)
    assert np.max(np.abs(err[:, N // 2])) < (1e-9 if precision == "fp64" else 1e-5)


def test_backward_time_step():
    w = W.ufg_plane_waves(16, 20, noise_eps=0.1)
    w.dt = -0.005
    check_run(w, 6)


@pytest.mark.parametrize("precision", ["mixed", "mixed_strict"])
def test_mixed_run_error_bound(precision):
    w = W.ufg_plane_waves(16, 64, noise_eps=1e-3, steps=20)
    g = run_gpu(w, w.steps, precision=precision)
    o = run_oracle(w, w.steps)
    # per right-hand side the FP32 error is ~1e-7 relative; it enters y through dt
    # times the ABM weights, over 3 start steps (8 H psi each) and 20 steps
    assert rel(g[0], o[0]) < 5e-6
    assert rel(g[1], o[1]) < 5e-6
    assert rel(g[2], o[2]) < 5e-6
    assert abs(g[3] - o[3]) / abs(o[3]) < 1e-6


# ------------------------------------------------------- full-size sample ----

def test_trap_vortex_full_size_rhs_sampled():
    # the full 32^3 x 2048-state workload: one right-hand side on the GPU; the oracle
    # checks sampled states one by one with densities built from all states
    w = W.named("trap32_vortex_fp64")
    psi = w.initial_state()
    with L.Context.from_workload(w) as ctx:
        got = ctx.rhs(psi, 0.25)
    p = oracle_params(w)
    n, nu = O.densities(p, psi)
    Wp, Dp = O.potentials(p, n, nu, 0.25)
    sample = [0, 1, 777, 1500, 2046, 2047]
    ps = p.with_(n_qp=len(sample))
    ref = -1j * O.apply_h(ps, Wp, Dp, psi[sample])
    assert rel(got[sample], ref) < TOL_FP64_RHS


def test_trap_vortex_full_size_invariants():
    w = W.named("trap32_vortex_fp64")
    with L.Context.from_workload(w) as ctx:
        ctx.set_state(w.initial_state(), 0.0, w.dt)
        E0, N0 = ctx.energy()
        ctx.step(10)
        E1, N1 = ctx.energy()
        psi = ctx.state()
    assert abs(N1 - N0) / N0 < 1e-9
    # state norms stay 1 to the integrator's truncation level
    norms = np.sum(np.abs(psi) ** 2, axis=(1, 2, 3, 4)) * w.a ** 3
    assert np.abs(norms - 1).max() < 1e-9


# ---------------------------------------------------------------- errors ----

def test_error_paths():
    w = W.ufg_plane_waves(8, 4)
    with L.Context.from_workload(w) as ctx:
        with pytest.raises(L.LiseError) as e:
            ctx.step(1, 0.005)
        assert e.value.status == L.ESTATE
        bad = w.initial_state()
        bad[1, 0, 2, 3, 4] = np.nan
        with pytest.raises(L.LiseError) as e:
            ctx.set_state(bad, 0.0, 0.005)
        assert e.value.status == L.ENONFINITE
        # the context stays usable after a rejected input
        ctx.set_state(w.initial_state(), 0.0, 0.005)
        with pytest.raises(L.LiseError) as e:
            ctx.step(1, 0.004)
        assert e.value.status == L.EINVAL
        with pytest.raises(L.LiseError) as e:
            ctx.set_state(w.initial_state(), 0.0, 0.0)
        assert e.value.status == L.EINVAL
        ctx.step(2)
        ctx.sync()


def test_nonfinite_density_reported():
    # a state that overflows |v|^2 in the density reduction is reported, not propagated
    w = W.ufg_plane_waves(8, 4)
    psi = w.initial_state()
    psi[0, 1] *= 1e200
    with L.Context.from_workload(w) as ctx:
        with pytest.raises(L.LiseError) as e:
            ctx.set_state(psi, 0.0, 0.005)
        assert e.value.status == L.ENONFINITE


def test_deterministic_bitwise():
    w = W.ufg_plane_waves(16, 40, noise_eps=0.05)
    a = run_gpu(w, 5)
    b = run_gpu(w, 5)
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])


# ------------------------------------------------------------ checkpoint ----

@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_strict"])
def test_checkpoint_bit_exact_resume(precision):
    w = W.ufg_plane_waves(16, 20, noise_eps=0.05)
    with L.Context.from_workload(w, precision=precision) as a:
        a.set_state(w.initial_state(), 0.0, w.dt)
        a.step(10)
        ref, t_ref = a.state(), a.t
    with L.Context.from_workload(w, precision=precision) as b:
        b.set_state(w.initial_state(), 0.0, w.dt)
        b.step(4)
        ck = b.checkpoint()
        b.step(6)
        assert np.array_equal(b.state(), ref)
    with L.Context.from_workload(w, precision=precision) as c:
        c.restore(ck)
        c.step(6)
        assert c.t == t_ref
        assert np.array_equal(c.state(), ref)


def test_checkpoint_rejects_other_shapes():
    w = W.ufg_plane_waves(8, 6)
    with L.Context.from_workload(w) as a:
        with pytest.raises(L.LiseError) as e:
            a.checkpoint()
        assert e.value.status == L.ESTATE
        a.set_state(w.initial_state(), 0.0, w.dt)
        ck = a.checkpoint()
    w2 = W.ufg_plane_waves(8, 7)
    with L.Context.from_workload(w2) as b:
        with pytest.raises(L.LiseError) as e:
            b.restore(np.concatenate([ck, np.zeros(1 << 16, np.uint8)]))
        assert e.value.status == L.EINVAL
    with L.Context.from_workload(w, precision="mixed") as b:
        with pytest.raises(L.LiseError) as e:
            b.restore(ck)
        assert e.value.status == L.EINVAL


# ------------------------------------------------------ mixed energy drift ----

def test_mixed_energy_drift_vs_fp64():
    # the driven 48^3 workload with 32 states, 400 steps: the energy of both mixed splits
    # stays within 1e-6 (relative) of the FP64 trajectory at every sample
    w = W.driven(48, 32, steps=400)
    E = {}
    for prec in ("fp64", "mixed", "mixed_strict"):
        with L.Context.from_workload(w, precision=prec) as ctx:
            ctx.set_state(w.initial_state(), 0.0, w.dt)
            e = [ctx.energy()[0]]
            for _ in range(8):
                ctx.step(50)
                e.append(ctx.energy()[0])
            E[prec] = np.array(e)
    for prec in ("mixed", "mixed_strict"):
        dev = np.max(np.abs(E[prec] - E["fp64"]) / np.abs(E["fp64"]))
        assert dev < 1e-6, (prec, dev)


# ---------------------------------------------------- trivial-phase removal ----

@pytest.mark.parametrize("N,precision,tol", [(16, "fp64", TOL_FP64_RHS), (16, "mixed", 2e-6),
                                             (12, "fp64", TOL_FP64_RHS), (20, "fp64", TOL_FP64_RHS),
                                             (48, "fp64", TOL_FP64_RHS)])
def test_rhs_phase_removal(N, precision, tol):
    n_qp = 7
    psi = random_state(N, n_qp, seed=21, kmax=5)
    kw = dict(alpha=1.1, beta=-0.5, mu=0.2, g=0.9)
    with L.Context(N, n_qp, precision=precision, remove_phase=True, **kw) as ctx:
        got = ctx.rhs(psi, 0.4)
    ref = O.rhs(O.Params(N, N, N, n_qp=n_qp, remove_phase=True, **kw), psi, 0.4)
    assert rel(got, ref) < tol


def test_run_phase_removal():
    w = W.ufg_plane_waves(12, 9, noise_eps=0.1, steps=8)
    with L.Context.from_workload(w, remove_phase=True) as ctx:
        ctx.set_state(w.initial_state(), 0.0, w.dt)
        ctx.step(w.steps)
        got = ctx.state()
        n, nu = ctx.densities()
    s = O.Solver(oracle_params(w, remove_phase=True))
    s.set_state(w.initial_state(), 0.0, w.dt)
    s.step(w.steps)
    assert rel(got, s.state()) < TOL_FP64_RUN
    on, onu = s.densities()
    assert rel(n, on) < TOL_FP64_RUN and rel(nu, onu) < TOL_FP64_RUN


def test_phase_removal_keeps_stationary_state():
    w = W.ufg_plane_waves(8, 24, noise_eps=0.0, delta0=0.5)
    U_, V_ = w.amps[:, 0], w.amps[:, 1]
    g_sc = -w.delta0 / (np.sum(U_ * V_) / (w.nxyz * w.a ** 3))
    with L.Context(8, 24, alpha=w.alpha, beta=w.beta, mu=w.mu, g=g_sc, remove_phase=True) as ctx:
        ctx.set_state(w.initial_state(), 0.0, 0.01)
        ctx.step(40)
        got = ctx.state()
    assert rel(got, w.initial_state()) < 1e-13


# -------------------------------------------- pairing coupling (Eqs. g0, geff_3D) ----

def test_rhs_density_dependent_renormalised_pairing():
    N, n_qp = 16, 6
    psi = random_state(N, n_qp, seed=41, kmax=5)
    kw = dict(alpha=1.0, beta=-0.5, mu=0.25, g=-1.2, pair_alpha=0.5, pair_n0=0.02, pair_lattice=True)
    with L.Context(N, n_qp, **kw) as ctx:
        got = ctx.rhs(psi, 0.0)
    ref = O.rhs(O.Params(N, N, N, n_qp=n_qp, **kw), psi, 0.0)
    assert rel(got, ref) < TOL_FP64_RHS


def test_run_density_dependent_renormalised_pairing():
    w = W.ufg_plane_waves(12, 10, noise_eps=0.2, g=-0.9, steps=6)
    n0 = 2 * np.sum(w.amps[:, 1] ** 2) / (w.nxyz * w.a ** 3)
    kw = dict(pair_alpha=0.4, pair_n0=n0, pair_lattice=True)
    with L.Context.from_workload(w, **kw) as ctx:
        ctx.set_state(w.initial_state(), 0.0, w.dt)
        ctx.step(w.steps)
        got = ctx.state()
        E, N = ctx.energy()
    s = O.Solver(oracle_params(w, **kw))
    s.set_state(w.initial_state(), 0.0, w.dt)
    s.step(w.steps)
    assert rel(got, s.state()) < TOL_FP64_RUN
    Eo, No = s.energy()
    assert E == pytest.approx(Eo, rel=1e-11)


# ------------------------------------- pairing coupling (Eq. geff, spherical cutoff) ----

def _u_loc(p, psi):
    nn, _ = O.densities(p, psi)
    u = 0.5 * p.beta * (3 * np.pi ** 2 * nn) ** (2.0 / 3.0)
    return u + (p.v_static if p.v_static is not None else 0.0)


def test_rhs_spherical_cutoff_pairing():
    # sites on both branches of Eq. geff (k_F^2 of either sign), a density-dependent g0
    N, n_qp = 16, 6
    psi = random_state(N, n_qp, seed=43, kmax=5)
    vs = np.random.default_rng(3).uniform(-1, 1, (N, N, N))
    kw = dict(alpha=1.1, beta=-0.5, mu=0.25, g=-1.2, pair_alpha=0.5, pair_n0=0.02, pair_ec=2.0)
    p = O.Params(N, N, N, n_qp=n_qp, v_static=vs, drive_A=0.02, drive_Omega=0.3, **kw)
    u = _u_loc(p, psi)
    assert (u < p.mu).sum() > 100 and (u > p.mu).sum() > 100
    with L.Context(N, n_qp, v_static=vs, drive_A=0.02, drive_Omega=0.3, **kw) as ctx:
        got = ctx.rhs(psi, 0.7)
    ref = O.rhs(p, psi, 0.7)
    assert rel(got, ref) < TOL_FP64_RHS
    assert maxabs_rel(got, ref) < TOL_FP64_ELEM


@pytest.mark.parametrize("precision,tol", [("fp64", TOL_FP64_RUN), ("mixed", 5e-6)])
def test_run_spherical_cutoff_pairing(precision, tol):
    # the driven workload in a trap: k_F^2 > 0, k_F^2 < 0 and empty-sphere (k_c^2 < 0) sites,
    # with the drive moving U_loc in time (graph replays read the drive from device memory)
    w = W.driven(12, 10, A=0.05, Omega=0.3, noise_eps=0.2, g=-0.9, steps=6)
    w.v_static = W.harmonic_trap(12, 0.15)
    kw = dict(pair_alpha=0.4, pair_n0=0.01, pair_ec=0.5)
    p = oracle_params(w, **kw)
    u = _u_loc(p, w.initial_state())
    assert (u < p.mu).sum() > 100 and (u > p.mu + 0.5).sum() > 100
    with L.Context.from_workload(w, precision=precision, **kw) as ctx:
        ctx.set_state(w.initial_state(), 0.0, w.dt)
        ctx.step(w.steps)
        got = ctx.state()
        E, _ = ctx.energy()
    s = O.Solver(p)
    s.set_state(w.initial_state(), 0.0, w.dt)
    s.step(w.steps)
    assert rel(got, s.state()) < tol
    Eo, _ = s.energy()
    assert E == pytest.approx(Eo, rel=1e-11 if precision == "fp64" else 1e-6)


# ------------------------------------------------------------ CUDA graphs ----

@pytest.mark.parametrize("workload", ["ufg", "drive"])
def test_graph_replay_matches_plain_launches(workload):
    # lise_step replays captured 4-step graphs; with per-launch profiling on it launches
    # every kernel itself.  Both must give the same bits (13 steps = 3 replays + 1 plain).
    w = W.ufg_plane_waves(16, 20, noise_eps=0.05) if workload == "ufg" else W.driven(16, 20, A=0.05)
    out = []
    for profiled in (False, True):
        with L.Context.from_workload(w) as ctx:
            ctx.set_state(w.initial_state(), 0.0, w.dt)
            if profiled:
                ctx.profile(True)
            ctx.step(13)
            ctx.step(8)  # graphs replayed again from another ring position
            out.append((ctx.state(), ctx.t))
    assert out[0][1] == out[1][1]
    assert np.array_equal(out[0][0], out[1][0])


# ------------------------------------------------------------ boost (Eq. kick) ----

def test_kick_parity():
    # evolve, boost with a smooth periodic profile plus a lattice momentum, evolve again
    w = W.ufg_plane_waves(16, 12, noise_eps=0.05)
    N = w.nx
    x = np.arange(N) * w.a
    L_ = N * w.a
    chi = (0.3 * np.sin(2 * np.pi * x / L_)[None, None, :] + 0.2 * np.cos(4 * np.pi * x / L_)[:, None, None]
           + (2 * np.pi / L_) * x[None, :, None])
    with L.Context.from_workload(w) as ctx:
        with pytest.raises(L.LiseError) as e:
            ctx.kick(chi)
        assert e.value.status == L.ESTATE
        ctx.set_state(w.initial_state(), 0.0, w.dt)
        ctx.step(4)
        ctx.kick(chi)
        ctx.step(5)
        got, t = ctx.state(), ctx.t
    s = O.Solver(oracle_params(w))
    s.set_state(w.initial_state(), 0.0, w.dt)
    s.step(4)
    s.kick(chi)
    s.step(5)
    assert t == pytest.approx(s.t, abs=1e-14)
    assert rel(got, s.state()) < TOL_FP64_RUN


# ------------------------------------------------------------ current density (Eq. j) ----

@pytest.mark.parametrize("N,n_qp,precision", [(16, 9, "fp64"), (12, 5, "fp64"), (32, 5, "mixed")])
def test_currents_parity(N, n_qp, precision):
    psi = random_state(N, n_qp, seed=21 + N)
    kw = dict(a=0.9, alpha=1.0, beta=-0.5, mu=0.3, g=0.7)
    with L.Context(N, n_qp, precision=precision, **kw) as ctx:
        with pytest.raises(L.LiseError) as e:
            ctx.currents()
        assert e.value.status == L.ESTATE
        ctx.set_state(psi, 0.0, 0.005)
        y = ctx.state()          # the state after the 3-step series start
        j = ctx.currents()
    ref = O.currents(O.Params(N, N, N, n_qp=n_qp, **kw), y)
    assert rel(j, ref) < 1e-12


# ------------------------------------------------------------ per-step renormalisation ----

@pytest.mark.parametrize("N", [16, 12])
def test_renormalize_parity(N):
    w = W.ufg_plane_waves(N, 20, noise_eps=0.3)
    w.dt = 0.02  # the plain ABM norm drift is visible at this step
    with L.Context.from_workload(w, renormalize=True) as ctx:
        ctx.set_state(w.initial_state(), 0.0, w.dt)
        ctx.step(10)
        got = ctx.state()
    norms = np.sum(np.abs(got) ** 2, axis=(1, 2, 3, 4)) * w.a ** 3
    assert np.max(np.abs(norms - 1)) < 1e-14
    s = O.Solver(oracle_params(w, renormalize=True))
    s.set_state(w.initial_state(), 0.0, w.dt)
    s.step(10)
    assert rel(got, s.state()) < TOL_FP64_RUN


# ------------------------------------------------------------ pencil batch autotuning ----

@pytest.mark.parametrize("N,precision", [(16, "fp64"), (32, "fp64"), (24, "mixed"), (48, "mixed")])
def test_pencil_batch_choice_is_bitwise_neutral(N, precision):
    w = W.ufg_plane_waves(N, 13, noise_eps=0.05)

    def run():
        with L.Context.from_workload(w, precision=precision) as ctx:
            ctx.set_state(w.initial_state(), 0.0, w.dt)
            ctx.step(5)
            return ctx.state()

    outs = {}
    for qb in (1, 2, 4):
        try:
            L.set_pencil_batch(N, precision, qb)
        except L.LiseError:
            continue  # variant not compiled for this lattice (shared memory)
        outs[qb] = run()
    L.set_pencil_batch(N, precision, 0)   # the next set_state tunes
    tuned = run()
    assert L.pencil_batch(N, precision) in outs
    for x in outs.values():
        assert np.array_equal(x, tuned)


@pytest.mark.parametrize("N,precision", [(16, "mixed"), (24, "mixed"), (32, "mixed"), (48, "mixed"), (64, "mixed"),
                                         (12, "fp64")])
def test_planes_per_block_choice_is_bitwise_neutral(N, precision):
    w = W.ufg_plane_waves(N, 13, noise_eps=0.05)

    def run():
        with L.Context.from_workload(w, precision=precision) as ctx:
            ctx.set_state(w.initial_state(), 0.0, w.dt)
            ctx.step(5)
            return ctx.state()

    outs = {}
    for pb in (1, 2, 4, 8, -1, -2, -4, -8):   # negative: whole lines in registers (FP32 path)
        try:
            L.set_planes_per_block(N, precision, pb)
        except L.LiseError:
            continue  # variant not compiled for this lattice
        outs[pb] = run()
    L.set_planes_per_block(N, precision, 0)   # the next set_state tunes
    tuned = run()
    assert len(outs) >= 2
    assert L.planes_per_block(N, precision) in outs
    for x in outs.values():
        assert np.array_equal(x, tuned)


# ------------------------------------------------------------ large lattices ----

def test_fp64_run_64_cubed():
    # the largest lattice: tensor-core kinetic operator with K = 64 (levels converted per
    # 16-deep step) in both kernels
    w = W.ufg_plane_waves(64, 3, noise_eps=0.05, steps=3)
    check_run(w, w.steps)


@pytest.mark.parametrize("N", [40, 64])
def test_mixed_run_large_lattices(N):
    w = W.ufg_plane_waves(N, 4, noise_eps=1e-3, steps=4)
    g = run_gpu(w, w.steps, precision="mixed")
    o = run_oracle(w, w.steps)
    assert rel(g[0], o[0]) < 5e-6
    assert abs(g[3] - o[3]) / abs(o[3]) < 1e-6


def test_mixed_strict_is_the_more_accurate_split():
    # the strict split keeps every ABM combination and density in FP64: its state after a
    # run is at least as close to the FP64 oracle as the default split's (both are limited
    # by the FP32 transforms); and it differs from the default split (different arithmetic)
    w = W.driven(24, 16, A=0.05, noise_eps=0.05, steps=30, precision="fp64")
    o = run_oracle(w, w.steps)
    errs = {}
    for prec in ("mixed", "mixed_strict"):
        g = run_gpu(w, w.steps, precision=prec)
        errs[prec] = rel(g[0], o[0])
        assert errs[prec] < 5e-6, (prec, errs[prec])
    assert errs["mixed_strict"] != errs["mixed"]
    assert errs["mixed_strict"] < 1.2 * errs["mixed"], errs
