"""Thin ctypes binding of liblise.so (include/lise.h): argument marshalling only.

Every step of the TDSLDA path runs in the CUDA library; this module converts
numpy arrays or CUDA tensors to pointers and status codes to exceptions.  If
the library cannot be loaded the import fails: there is no fallback.

State arrays are complex128 of shape (n_qp, 2, N, N, N) (component 0 = u,
1 = v; index order z, y, x), densities have shape (N, N, N).
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblise.so")

FP64 = 0
MIXED = 1
MIXED_STRICT = 2
PRECISIONS = {"fp64": FP64, "mixed": MIXED, "mixed_strict": MIXED_STRICT}

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, ESTATE, EEXCHANGE = range(8)
ADMIT_FIFO, ADMIT_FIRST_FIT = 0, 1
KC_PLANES, KC_PENCILS, KC_REDUCE, KC_POINTWISE, KC_COUNT = range(5)


class LiseError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} (status {status})")


class _Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double),
                ("n_qp", C.c_int), ("alpha", C.c_double), ("beta", C.c_double),
                ("mu", C.c_double), ("g", C.c_double), ("v_static", C.c_void_p),
                ("drive_A", C.c_double), ("drive_Omega", C.c_double), ("precision", C.c_int),
                ("device", C.c_int), ("hbm_budget_bytes", C.c_size_t), ("stream", C.c_void_p),
                ("remove_phase", C.c_int), ("pair_alpha", C.c_double), ("pair_n0", C.c_double),
                ("pair_lattice", C.c_int), ("renormalize", C.c_int), ("pair_ec", C.c_double)]


# lise_exchange_fn and lise_shard (sharded densities)
EXCHANGE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_long, C.c_int, C.c_int,
                          C.c_int)


class _Shard(C.Structure):
    _fields_ = [("group_size", C.c_int), ("first_group", C.c_int), ("n_groups_all", C.c_int),
                ("exchange", EXCHANGE_FN), ("user", C.c_void_p), ("on_device", C.c_int), ("capturable", C.c_int)]


# Exported functions with their ctypes signatures (mirrors include/lise.h).
SIGNATURES = {
    "lise_footprint_bytes": (C.c_size_t, [C.c_void_p]),
    "lise_create": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lise_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_double]),
    "lise_set_state_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_double]),
    "lise_kick": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lise_currents": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lise_pencil_batch": (C.c_int, [C.c_int, C.c_int]),
    "lise_set_pencil_batch": (C.c_int, [C.c_int, C.c_int, C.c_int]),
    "lise_planes_per_block": (C.c_int, [C.c_int, C.c_int]),
    "lise_set_planes_per_block": (C.c_int, [C.c_int, C.c_int, C.c_int]),
    "lise_step": (C.c_int, [C.c_void_p, C.c_int, C.c_double]),
    "lise_get_state": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lise_get_state_device": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lise_get_time": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "lise_densities": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "lise_energy": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "lise_rhs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]),
    "lise_sync": (C.c_int, [C.c_void_p]),
    "lise_set_wait_limit": (C.c_int, [C.c_void_p, C.c_long]),
    "lise_set_shard": (C.c_int, [C.c_void_p, C.c_void_p]),
    "lise_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "lise_profile_read": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_long), C.POINTER(C.c_double)]),
    "lise_kernel_class_name": (C.c_char_p, [C.c_int]),
    "lise_strerror": (C.c_char_p, [C.c_int]),
    "lise_destroy": (None, [C.c_void_p]),
    "lise_rhs_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]),
    "lise_measure_fp64_peak": (C.c_int, [C.c_int, C.POINTER(C.c_double)]),
    "lise_checkpoint_bytes": (C.c_size_t, [C.c_void_p]),
    "lise_checkpoint_save": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "lise_checkpoint_load": (C.c_int, [C.c_void_p, C.c_void_p, C.c_size_t]),
    "lise_batch_create": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "lise_batch_step": (C.c_int, [C.c_void_p, C.c_int]),
    "lise_batch_sync": (C.c_int, [C.c_void_p]),
    "lise_batch_destroy": (None, [C.c_void_p]),
    "lise_server_create": (C.c_int, [C.c_int, C.c_size_t, C.c_int, C.c_int, C.c_void_p]),
    "lise_server_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_int,
                                     C.POINTER(C.c_long)]),
    "lise_server_wait": (C.c_int, [C.c_void_p, C.c_long, C.c_void_p, C.c_void_p]),
    "lise_server_submit_borrowed": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                              C.c_double, C.c_int, C.POINTER(C.c_long)]),
    "lise_server_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_size_t), C.POINTER(C.c_int)]),
    "lise_server_poll": (C.c_int, [C.c_void_p, C.c_long, C.POINTER(C.c_int)]),
    "lise_server_set_admission": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "lise_server_set_batching": (C.c_int, [C.c_void_p, C.c_int]),
    "lise_server_destroy": (None, [C.c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load liblise.so (raises OSError if it is missing or does not load)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise OSError(f"liblise.so not built at {path}; run paper_2009_00745_b300/build.py")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(status: int) -> str:
    return load().lise_strerror(int(status)).decode()


def _check(rc, where):
    if rc != OK:
        raise LiseError(rc, where)


def _params(N, n_qp, a, alpha, beta, mu, g, v_static, drive_A, drive_Omega, precision, device,
            hbm_budget_bytes, stream, remove_phase=False, pair_alpha=0.0, pair_n0=1.0, pair_lattice=False,
            renormalize=False, pair_ec=0.0):
    prec = PRECISIONS.get(precision, precision)
    vs = None
    if v_static is not None:
        vs = np.ascontiguousarray(v_static, dtype=np.float64).reshape(-1)
        if vs.size != N ** 3:
            raise ValueError("v_static must hold N^3 values")
    p = _Params(N, N, N, float(a), int(n_qp), float(alpha), float(beta), float(mu), float(g),
                None if vs is None else vs.ctypes.data, float(drive_A), float(drive_Omega),
                int(prec), int(device), int(hbm_budget_bytes), stream, int(bool(remove_phase)),
                float(pair_alpha), float(pair_n0), int(bool(pair_lattice)), int(bool(renormalize)),
                float(pair_ec))
    return p, vs


def pencil_batch(N, precision="fp64") -> int:
    """States per batch the pencils kernel uses for this lattice and precision (tuned or default)."""
    return int(load().lise_pencil_batch(int(N), PRECISIONS[precision]))


def set_pencil_batch(N, precision="fp64", qb=0):
    """Force the pencils batch size (1 for the FP64 tensor-core kernels, 2 or 4), or qb = 0 to
    re-tune at the next set_state."""
    _check(load().lise_set_pencil_batch(int(N), PRECISIONS[precision], int(qb)),
           "lise_set_pencil_batch")


def measure_fp64_peak(device=0) -> float:
    """FP64 FMA throughput of the device (TFLOP/s) from the library's probe kernel."""
    t = C.c_double()
    _check(load().lise_measure_fp64_peak(int(device), C.byref(t)), "lise_measure_fp64_peak")
    return t.value


def planes_per_block(N, precision="mixed") -> int:
    """Planes per block of the FFT planes kernel for this lattice and precision (0: tensor-core kernel;
    negative: the register-line variant with -pb planes per block)."""
    return int(load().lise_planes_per_block(int(N), PRECISIONS[precision]))


def set_planes_per_block(N, precision="mixed", pb=0):
    """Force the FFT planes kernel's variant, or 0 to re-tune: 1, 2, 4, 8 planes per block of the
    shared-memory kernel, -1, -2, -4, -8 of the register-line kernel (where compiled)."""
    _check(load().lise_set_planes_per_block(int(N), PRECISIONS[precision], int(pb)), "lise_set_planes_per_block")


def footprint_bytes(N, n_qp, precision="fp64", **kw) -> int:
    p, _ = _params(N, n_qp, kw.get("a", 1.0), kw.get("alpha", 1.0), kw.get("beta", 0.0),
                   kw.get("mu", 0.0), kw.get("g", 0.0), None, 0.0, 0.0, precision, 0, 0, None)
    return int(load().lise_footprint_bytes(C.byref(p)))


def _ptr(x, dtype=np.complex128, count=None, writable=False):
    """(pointer, is_device, keepalive) for a numpy array or a CUDA tensor."""
    if hasattr(x, "data_ptr") and hasattr(x, "is_cuda"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if count is not None and x.numel() * x.element_size() != count * np.dtype(dtype).itemsize:
            raise ValueError("tensor has the wrong size")
        return x.data_ptr(), bool(x.is_cuda), x
    a = np.asarray(x)
    if a.dtype != dtype or not a.flags.c_contiguous:
        if writable:
            raise ValueError(f"output array must be C-contiguous {np.dtype(dtype)}")
        a = np.ascontiguousarray(a, dtype=dtype)
    if count is not None and a.size != count:
        raise ValueError(f"array has {a.size} elements, expected {count}")
    return a.ctypes.data, False, a


class Context:
    """One TDSLDA evolution on one GPU (a lise_ctx)."""

    def __init__(self, N, n_qp, *, a=1.0, alpha=1.0, beta=0.0, mu=0.0, g=0.0, v_static=None,
                 drive_A=0.0, drive_Omega=0.0, precision="fp64", device=0, hbm_budget_bytes=0,
                 stream=None, remove_phase=False, pair_alpha=0.0, pair_n0=1.0, pair_lattice=False,
                 renormalize=False, pair_ec=0.0):
        self.N, self.n_qp = int(N), int(n_qp)
        self._p, self._vs = _params(N, n_qp, a, alpha, beta, mu, g, v_static, drive_A, drive_Omega,
                                    precision, device, hbm_budget_bytes, stream, remove_phase, pair_alpha,
                                    pair_n0, pair_lattice, renormalize, pair_ec)
        h = C.c_void_p()
        _check(load().lise_create(C.byref(self._p), C.byref(h)), "lise_create")
        self._h = h
        self.dt = None

    @classmethod
    def from_workload(cls, w, **kw):
        return cls(w.nx, w.n_qp, a=w.a, alpha=w.alpha, beta=w.beta, mu=w.mu, g=w.g,
                   v_static=w.v_static, drive_A=w.drive_A, drive_Omega=w.drive_Omega,
                   precision=kw.pop("precision", w.precision), **kw)

    @property
    def shape(self):
        return (self.n_qp, 2, self.N, self.N, self.N)

    @property
    def count(self):
        return self.n_qp * 2 * self.N ** 3

    def close(self):
        if getattr(self, "_h", None):
            load().lise_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_state(self, psi, t0, dt):
        ptr, dev, keep = _ptr(psi, count=self.count)
        fn = load().lise_set_state_device if dev else load().lise_set_state
        _check(fn(self._h, ptr, float(t0), float(dt)), "lise_set_state")
        self.dt = float(dt)

    def currents(self):
        """Current density of Eq. j of the current state: array [3][z][y][x] (x, y, z components)."""
        out = np.empty((3, self.N, self.N, self.N))
        _check(load().lise_currents(self._h, out.ctypes.data), "lise_currents")
        return out

    def kick(self, chi):
        """Eq. kick on the current state (u e^{i chi}, v e^{-i chi}), then a new series start."""
        chi = np.ascontiguousarray(chi, dtype=np.float64)
        if chi.size != self.N ** 3:
            raise ValueError(f"chi has {chi.size} values, expected {self.N ** 3}")
        _check(load().lise_kick(self._h, chi.ctypes.data), "lise_kick")

    def step(self, n_steps, dt=None):
        _check(load().lise_step(self._h, int(n_steps), float(self.dt if dt is None else dt)), "lise_step")

    def state(self, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=np.complex128)
        ptr, dev, _ = _ptr(out, count=self.count, writable=True)
        fn = load().lise_get_state_device if dev else load().lise_get_state
        _check(fn(self._h, ptr), "lise_get_state")
        return out

    @property
    def t(self):
        t = C.c_double()
        _check(load().lise_get_time(self._h, C.byref(t)), "lise_get_time")
        return t.value

    def densities(self):
        n = np.empty((self.N,) * 3)
        nu = np.empty((self.N,) * 3, dtype=np.complex128)
        _check(load().lise_densities(self._h, n.ctypes.data, nu.ctypes.data), "lise_densities")
        return n, nu

    def energy(self):
        E, Nn = C.c_double(), C.c_double()
        _check(load().lise_energy(self._h, C.byref(E), C.byref(Nn)), "lise_energy")
        return E.value, Nn.value

    def rhs(self, psi, t):
        ptr, _, keep = _ptr(psi, count=self.count)
        out = np.empty(self.shape, dtype=np.complex128)
        _check(load().lise_rhs(self._h, ptr, float(t), out.ctypes.data), "lise_rhs")
        return out

    def profile(self, enable=True):
        """Record a CUDA event pair around every kernel launch (clears old records)."""
        _check(load().lise_profile(self._h, int(bool(enable))), "lise_profile")

    def profile_read(self):
        """{class name: (launches, total device ms)} since profiling was enabled."""
        out = {}
        for k in range(KC_COUNT):
            n, ms = C.c_long(), C.c_double()
            _check(load().lise_profile_read(self._h, k, C.byref(n), C.byref(ms)), "lise_profile_read")
            out[load().lise_kernel_class_name(k).decode()] = (n.value, ms.value)
        return out

    def checkpoint(self):
        """The full ABM history as bytes (a bit-exact restart point)."""
        n = int(load().lise_checkpoint_bytes(self._h))
        buf = np.empty(n, dtype=np.uint8)
        _check(load().lise_checkpoint_save(self._h, buf.ctypes.data, n), "lise_checkpoint_save")
        return buf

    def restore(self, buf):
        """Load a checkpoint taken from a context with the same lattice, states and precision."""
        b = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(load().lise_checkpoint_load(self._h, b.ctypes.data, b.size), "lise_checkpoint_load")
        self.dt = float(np.frombuffer(b[32:40].tobytes(), dtype=np.float64)[0])  # header: t at 24, dt at 32

    def sync(self):
        _check(load().lise_sync(self._h), "lise_sync")

    def set_shard(self, group_size, first_group=0, n_groups_all=None, exchange=None, on_device=False,
                  capturable=False):
        """Sharded densities (lise_set_shard): this context holds n_qp of the evolution's states,
        its density groups are first_group .. of n_groups_all groups of group_size states.
        exchange(parts, on_device, stream, nxyz, first_group, n_local, n_groups_all) fills the
        other shards' groups of the partial-sum block at address `parts` (see shard.py); an
        exception in it fails the library call with EEXCHANGE.  Call before set_state."""
        if n_groups_all is None:  # (a group size < 1 is left to the library to reject)
            n_groups_all = first_group + (-(-self.n_qp // int(group_size)) if int(group_size) > 0 else 0)
        if exchange is None:
            cb = EXCHANGE_FN()
        else:
            def cb_py(user, parts, on_dev, stream, nxyz, first, nloc, nall):
                try:
                    exchange(parts, bool(on_dev), stream, nxyz, first, nloc, nall)
                    return 0
                except Exception:
                    import traceback
                    traceback.print_exc()
                    return 1
            cb = EXCHANGE_FN(cb_py)
        sh = _Shard(int(group_size), int(first_group), int(n_groups_all), cb, None, int(bool(on_device)),
                    int(bool(capturable)))
        _check(load().lise_set_shard(self._h, C.byref(sh)), "lise_set_shard")
        self._exchange_cb = cb  # kept alive while the library may call it

    def set_wait_limit(self, polls):
        """Polls before a bounded device wait gives up (> 0), 0 = give up at once, < 0 = default."""
        _check(load().lise_set_wait_limit(self._h, int(polls)), "lise_set_wait_limit")


class Batch:
    """Several contexts (FP32 compute precision, after set_state) stepped together in shared
    launches (lise_batch_*).  Use the contexts only through the batch until sync() or close()."""

    def __init__(self, contexts):
        self._ctxs = list(contexts)
        arr = (C.c_void_p * len(self._ctxs))(*[c._h.value for c in self._ctxs])
        h = C.c_void_p()
        _check(load().lise_batch_create(arr, len(self._ctxs), C.byref(h)), "lise_batch_create")
        self._h = h

    def step(self, n_steps):
        _check(load().lise_batch_step(self._h, int(n_steps)), "lise_batch_step")

    def sync(self):
        _check(load().lise_batch_sync(self._h), "lise_batch_sync")

    def close(self):
        if getattr(self, "_h", None):
            load().lise_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class RequestInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("submit_s", C.c_double), ("admit_s", C.c_double),
                ("done_s", C.c_double), ("t", C.c_double), ("E", C.c_double), ("N", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Server:
    """Request loop over one GPU (lise_server_*): admission under an HBM budget,
    overlapping step chunks of the active requests."""

    def __init__(self, hbm_budget_bytes, *, device=0, max_active=8, steps_per_turn=4):
        h = C.c_void_p()
        _check(load().lise_server_create(int(device), int(hbm_budget_bytes), int(max_active),
                                         int(steps_per_turn), C.byref(h)), "lise_server_create")
        self._h = h
        self._shapes = {}
        self._borrowed = {}  # id -> (input, output) arrays the server reads/writes until wait()

    def submit(self, N, n_qp, psi, t0, dt, n_steps, *, a=1.0, alpha=1.0, beta=0.0, mu=0.0, g=0.0,
               v_static=None, drive_A=0.0, drive_Omega=0.0, precision="fp64", copy=True, out=None):
        """Queue one evolution.  copy=True: the server copies psi now.  copy=False: the
        server reads psi at admission and writes the final state into `out` (None: no
        state is returned); both arrays must stay untouched until wait()."""
        p, vs = _params(N, n_qp, a, alpha, beta, mu, g, v_static, drive_A, drive_Omega, precision, 0, 0, None)
        ptr, dev, keep = _ptr(psi, count=n_qp * 2 * N ** 3)
        if dev:
            raise ValueError("the server takes host states")
        rid = C.c_long()
        if copy:
            _check(load().lise_server_submit(self._h, C.byref(p), ptr, float(t0), float(dt), int(n_steps),
                                             C.byref(rid)), "lise_server_submit")
        else:
            optr = None
            if out is not None:
                optr, odev, _ = _ptr(out, count=n_qp * 2 * N ** 3, writable=True)
                if odev:
                    raise ValueError("the server takes host states")
            _check(load().lise_server_submit_borrowed(self._h, C.byref(p), ptr, optr, float(t0), float(dt),
                                                      int(n_steps), C.byref(rid)), "lise_server_submit_borrowed")
            self._borrowed[rid.value] = (keep, out)
        self._shapes[rid.value] = (n_qp, 2, N, N, N)
        return rid.value

    def submit_workload(self, w, psi=None, n_steps=None, precision=None):
        return self.submit(w.nx, w.n_qp, w.initial_state() if psi is None else psi, 0.0, w.dt,
                           w.steps if n_steps is None else n_steps, a=w.a, alpha=w.alpha, beta=w.beta,
                           mu=w.mu, g=w.g, v_static=w.v_static, drive_A=w.drive_A,
                           drive_Omega=w.drive_Omega, precision=precision or w.precision)

    def wait(self, rid, want_state=True):
        """(final state or None, info dict).  For copy=False submissions the state is the
        `out` array given at submit (None if none was given)."""
        shape = self._shapes.pop(rid)
        borrowed = self._borrowed.pop(rid, None)
        out = None
        if borrowed is None and want_state:
            out = np.empty(shape, dtype=np.complex128)
        info = RequestInfo()
        rc = load().lise_server_wait(self._h, int(rid), None if out is None else out.ctypes.data,
                                     C.byref(info))
        _check(rc, "lise_server_wait")
        if borrowed is not None:
            out = borrowed[1]
        return out, info.as_dict()

    def poll(self, rid):
        """True if request rid has finished (wait() then returns at once)."""
        d = C.c_int()
        _check(load().lise_server_poll(self._h, int(rid), C.byref(d)), "lise_server_poll")
        return bool(d.value)

    def set_admission(self, policy="fifo", max_skips=0):
        """'fifo' (arrival order) or 'first_fit' (a request may be passed over at most max_skips times)."""
        code = {"fifo": ADMIT_FIFO, "first_fit": ADMIT_FIRST_FIT}[policy]
        _check(load().lise_server_set_admission(self._h, code, int(max_skips)), "lise_server_set_admission")

    def set_batching(self, enable=True):
        """Step the active mixed-precision requests together in shared launches (before submitting)."""
        _check(load().lise_server_set_batching(self._h, int(bool(enable))), "lise_server_set_batching")

    def stats(self):
        u, a = C.c_size_t(), C.c_int()
        _check(load().lise_server_stats(self._h, C.byref(u), C.byref(a)), "lise_server_stats")
        return {"peak_used_bytes": u.value, "peak_active": a.value}

    def close(self):
        if getattr(self, "_h", None):
            load().lise_server_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
