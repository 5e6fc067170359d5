"""Throughput benchmark of the TDSLDA step (qp*site*steps/s) on B300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl reference]

A "step" is one Adams-Bashforth-Milne step (Eqs. p, m, c, y of arXiv:2009.00745:
two right-hand sides, each a kinetic operator, a BdG apply and a density
reduction) over all quasiparticle states of the workload.  Default workload:
32^3 lattice, 2048 states in a harmonic trap with a vortex phase, FP64
(trap32_vortex_fp64).  Inputs are synthetic and seeded (workloads.py).

value        device time of K steps with the state resident in HBM (CUDA events
             on the context's stream, W warm-up steps first).  The state and ABM
             history (~21 GB in FP64) are far larger than L2, so no flush.
e2e          the same metric through the C ABI with host buffers: lise_set_state
             from pinned host memory (including the start procedure), K steps,
             lise_get_state back to pinned host memory and lise_energy.
roofline     the kernel class with the largest share of device time (per-launch
             CUDA events).  frac: the fully fused step's algorithmic bytes
             (FUSED_BYTES per state and site, over the two pencils launches of a
             step) per launch over the mean launch time, against the measured HBM
             copy bandwidth; step: the same bytes over the whole step time;
             fp64_pipe (FP64 path): the FP64 flops the pencils kernel executes
             against the FP64 FMA peak measured by the library's probe kernel;
             traffic: DRAM bytes per launch from the committed ncu summary
             (profiles/traffic.json) when it was taken on the current sources.
pair         the metric's comparison: the driven 48^3 x 4096 workload timed in
             FP64 and in the mixed path (same K and W), mixed / FP64, and the mixed
             path's energy against the FP64 trajectory over 100 steps.
cpu_baseline the FP64 CPU oracle on a bounded sample of the same workload, on the
             host cores (thread count reported).
clocks       SM clocks and throttle reasons sampled during the timed region.
gpu_launches the library's kernel launches inside the timed region.
--impl reference times the FP64 CPU oracle instead (a deliberately plain program
on the host cores).  Multi-GPU (torchrun): every rank runs an independent replica
("replicas only"; the single-GPU path has no exchange step), value = total units /
max time.  --drift, --serve and --batch run the other measurements (see their
functions).
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "qp·site·steps/s, FP64 vs mixed at ≤1e-6 rel energy drift; p50/p99 latency"
UNIT = "qp·site·steps/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
HBM_FALLBACK_GBS = 6400.0
# Algorithmic HBM bytes per (state, site, step) of a fully fused step (each kinetic
# operator in one on-chip pass): 15 state-array passes of 32 B in FP64 (the corrector
# launch reads m, Q, R and writes y_{n+1}, p - c; the derivative/predictor launch reads
# y_{n+1}, y_n, y'_n..y'_{n-2}, p - c and writes y'_{n+1}, m, Q, R), 448 B with the
# mixed path's complex64 m and transform intermediates.  Keys: mixed (False/True).
FUSED_BYTES = {False: 480, True: 448}


def log2(n):
    return math.log2(n)


def algorithmic_per_qp_site(N, mixed, strict=False):
    """Algorithmic flops and HBM bytes per (state, site) of each kernel class
    for one ABM step (two right-hand sides), for the kernels as designed:

    planes     read the operand, write T_xy (both components);
    pencils    corrector launch: read m, T_xy, Q, R; write y_{n+1}, p - c.
               FP64 derivative/predictor launch: read y_{n+1}, T_xy, y_n,
               y'_n, y'_{n-1}, y'_{n-2}, p - c; write y'_{n+1}, m, Q, R.
               Mixed derivative launch: read y_{n+1}, T_xy; write y'_{n+1}.
    pointwise  (mixed only) predictor: read y_{n+1}, y_n, y'_{n+1}..y'_{n-2},
               p - c; write m, Q, R.
    complex128 = 16 B per component.  The states y and Q are complex128; T_xy,
    m, the y' ring, R and p - c are kept in the compute precision (complex64
    in the mixed path; R and p - c complex128 in its strict split).
    FFT convention: 5 n log2 n real flops per complex length-n transform.

    FP64 path on lattices with N % 16 == 0: the kinetic operator runs on the
    bf16 tensor cores (exact digit products, 28 digit pairs, K = N per axis),
    so "flops" of planes are its bf16 tensor flops and "flops" of pencils the
    FP64 flops its kernels execute (an FMA counts 2; work done exactly in
    integers -- T_z + T_xy, the derivative sums of Eqs. p, c -- is not counted):
      corrector  per real: BdG 3 FMA, y_{n+1} 1 FMA, p - c 1 FMA               -> 10
                 densities 3 x 2 FMA per (state, site)                          -> 12
      deriv/pred per real: BdG 3 FMA, P = hf + h/48 sp 1 + 1 FMA (the halving of
                 hf is an exponent decrement), Q 1 FMA, m 1 FMA                 -> 13
                 densities                                                      -> 12
    per (state, site): 2 components x 2 reals."""
    L = log2(N)
    c16, cr = 16, (8 if mixed else 16)   # complex128 / compute-precision component
    hr = 16 if (strict or not mixed) else 8  # R and p - c
    tensor = (not mixed) and N % 16 == 0
    planes_bytes = 2 * (cr + cr) + 2 * (c16 + cr)          # operand m, then operand y_{n+1}
    correct_bytes = 2 * (cr + cr + c16 + hr) + 2 * (c16 + hr)
    fft_bdg = 2 * (2 * 5 * L + 4) + 24                     # z fwd+inv + multiply/add, BdG apply
    planes_flops = 2 * 2 * (2 * 2 * 5 * L + 3)              # 2 launches x 2 comps: 2D fwd+inv, multiply
    predict_flops = 92 + 13                                 # Eq. p/m, Q, R, densities of m
    if mixed:
        deriv_bytes = 2 * (c16 + cr) + 2 * cr
        predict_bytes = 2 * (2 * c16 + 4 * cr + hr) + 2 * (cr + c16 + hr)
        pencils_flops = 2 * fft_bdg + (16 + 13)
        pointwise = {"flops": predict_flops, "bytes": predict_bytes, "launches_per_step": 1}
    else:
        deriv_bytes = 2 * (2 * c16 + 5 * cr) + 2 * (c16 + 3 * cr)
        pencils_flops = 2 * fft_bdg + (16 + 13) + predict_flops
        pointwise = {"flops": 0.0, "bytes": 0, "launches_per_step": 0}
    out = {
        "planes": {"flops": planes_flops, "bytes": planes_bytes, "launches_per_step": 2},
        "pencils": {"flops": pencils_flops, "bytes": correct_bytes + deriv_bytes, "launches_per_step": 2},
        "pointwise": pointwise,
    }
    if tensor:
        mma = 2 * 2 * N * 28 * 2          # bf16 flops per (state, site) and axis: 2 comps x re/im x K x pairs
        out["planes"].update({"flops": 2 * 2 * mma, "kind": "bf16 tensor"})
        out["pencils"].update({"flops": 4 * 10 + 12 + 4 * 13 + 12, "kind": "fp64", "tensor_flops": 2 * mma})
    return out


def read_peaks():
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2009_00745_b300", "csrc")
    for name in ("lise_fft.cuh", "lise_ozaki.cuh", "lise_kernels.cuh", "lise_kernels.cu"):  # the kernels' sources
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload, kernel, precision):
    """dram bytes per launch from the committed ncu summary, if it was taken on the
    current kernel sources in this precision (profiles/traffic.json: {workload: {kernel: {...}}},
    or {"workload@precision": {...}} for a workload measured in a precision other than its own)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(f"{workload}@{precision}", d.get(workload, {}))[kernel]
        if e.get("source_hash") != kernel_source_hash() or e.get("precision") != precision:
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def whole_job_value(ms_local, units_per_rank, world, device="cpu"):
    """Replicas: every rank times the same amount of work; the job time is the
    maximum over ranks and value = world * units / job time.  Returns
    (value, job_ms)."""
    ms = float(ms_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * float(units_per_rank) / (ms / 1e3), ms


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def oracle_sample_rate(w, n_sample, steps, warmup):
    """The FP64 CPU oracle as it stands on the first n_sample states of workload w:
    start procedure (untimed), warmup ABM steps (untimed), then `steps` timed ABM
    steps.  Returns (qp*site*steps/s, seconds, threads)."""
    from oracle import oracle as O
    p = O.Params(w.nx, w.ny, w.nz, a=w.a, n_qp=n_sample, alpha=w.alpha, beta=w.beta, mu=w.mu, g=w.g,
                 v_static=w.v_static, drive_A=w.drive_A, drive_Omega=w.drive_Omega)
    s = O.Solver(p)
    s.set_state(w.initial_state(0, n_sample), 0.0, w.dt)
    if warmup:
        s.step(warmup)
    t0 = time.perf_counter()
    s.step(steps)
    dt = time.perf_counter() - t0
    return n_sample * w.nxyz * steps / dt, dt, O.num_threads()


def run_reference(args, w):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    n_sample = args.ref_states
    rate, secs, thr = oracle_sample_rate(w, n_sample, args.steps, args.warmup)
    sample = (f"first {n_sample} of {w.n_qp} states of {w.name} ({w.nx}^3), start procedure untimed, "
              f"{args.warmup} warm-up + {args.steps} timed ABM steps")
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(w, args),
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_drift(args, w):
    """Both mixed splits against FP64 on the same workload: K ABM steps each, the
    energy sampled every --drift-every steps.  Reports, for LISE_MIXED and
    LISE_MIXED_STRICT, max_t |E_mixed(t) - E_FP64(t)| / |E_FP64(t)| (the energy of a
    truncated set of states is not an invariant, so the FP64 trajectory is the
    reference) and the final relative errors of psi, n, nu."""
    import numpy as np
    import torch
    from paper_2009_00745_b300 import lise as L
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    psi_host = torch.empty((w.n_qp, 2, w.nz, w.ny, w.nx), dtype=torch.complex128, pin_memory=True)
    w.initial_state(out=psi_host.numpy())
    K, every = args.steps, args.drift_every
    out = {}
    for prec in ("fp64", "mixed", "mixed_strict"):
        t0 = time.perf_counter()
        with L.Context.from_workload(w, precision=prec, device=local) as ctx:
            ctx.set_state(psi_host.numpy(), 0.0, w.dt)
            E = [ctx.energy()]
            done = 0
            while done < K:
                k = min(every, K - done)
                ctx.step(k)
                done += k
                E.append(ctx.energy())
            psi = ctx.state()
            n, nu = ctx.densities()
        out[prec] = {"E": np.array([e[0] for e in E]), "N": np.array([e[1] for e in E]), "psi": psi, "n": n,
                     "nu": nu, "seconds": time.perf_counter() - t0}
    f = out["fp64"]
    rel = lambda a, b: float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))
    line = {"mode": "drift", "workload": w.name, "lattice": f"{w.nx}^3", "n_qp": w.n_qp, "steps": K,
            "dt": w.dt, "sample_every": every,
            "fp64_energy_change": float(abs(f["E"][-1] - f["E"][0]) / abs(f["E"][0])),
            "fp64_N_change": float(abs(f["N"][-1] - f["N"][0]) / abs(f["N"][0])),
            "seconds": {k: v["seconds"] for k, v in out.items()}}
    for prec in ("mixed", "mixed_strict"):
        m = out[prec]
        line[prec] = {"max_rel_energy_dev_vs_fp64": float(np.max(np.abs(m["E"] - f["E"]) / np.abs(f["E"]))),
                      "rel_err_psi": rel(m["psi"], f["psi"]), "rel_err_n": rel(m["n"], f["n"]),
                      "rel_err_nu": rel(m["nu"], f["nu"]),
                      "max_rel_N_dev_vs_fp64": float(np.max(np.abs(m["N"] - f["N"]) / np.abs(f["N"])))}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """A Poisson stream of evolution requests through the serving loop.

    Requests arrive at --serve-rate per second (exponential gaps, seed 11); each
    draws a lattice from {16, 24, 32, 48}^3 and a state count uniform in
    [256, 4096], and runs 100 mixed-precision ABM steps; the server admits them
    under a 150 GB budget.  Each request evolves the first n_qp states of its
    lattice's 4096-state homogeneous BCS workload (built before the clock starts).
    Latency = done - arrival (arrival = the scheduled Poisson time).  Every request is stepped on
    its own context and stream; with --serve-batching the active requests of each lattice size are
    stepped together in shared launches (the server's batching)."""
    import numpy as np
    from paper_2009_00745_b300 import lise as L
    from paper_2009_00745_b300 import workloads as Wl
    rng = np.random.default_rng(11)
    R = args.serve_requests
    gaps = rng.exponential(1.0 / args.serve_rate, R)
    arrivals = np.cumsum(gaps) - gaps[0]
    lattices = rng.choice([16, 24, 32, 48], R)
    nqps = rng.integers(256, 4097, R)
    base = {}
    for n in sorted(set(int(x) for x in lattices)):
        w = Wl.ufg_plane_waves(n, 4096, noise_eps=1e-3, precision="mixed", steps=args.serve_steps)
        base[n] = (w, w.initial_state())
    budget = int(args.serve_budget_gb * 1e9)
    lag, sub_host, ids = [], [], []
    with L.Server(budget, max_active=args.serve_max_active, steps_per_turn=args.serve_turn) as srv:
        if args.serve_batching:
            srv.set_batching(True)
        t0 = time.perf_counter()
        for i in range(R):
            delay = t0 + arrivals[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            w, psi = base[int(lattices[i])]
            n_qp = int(nqps[i])
            ts = time.perf_counter()
            lag.append(ts - (t0 + arrivals[i]))
            ids.append(srv.submit(w.nx, n_qp, psi[:n_qp], 0.0, w.dt, args.serve_steps, a=w.a, alpha=w.alpha,
                                  beta=w.beta, mu=w.mu, g=w.g, precision="mixed", copy=False))
        infos = [srv.wait(i, want_state=False)[1] for i in ids]
        st = srv.stats()
    lat = np.array([inf["done_s"] - inf["submit_s"] + lg for inf, lg in zip(infos, lag)])
    queue = np.array([inf["admit_s"] - inf["submit_s"] + lg for inf, lg in zip(infos, lag)])
    units = sum(float(n) * int(l) ** 3 * args.serve_steps for n, l in zip(nqps, lattices))
    makespan = max(inf["done_s"] for inf in infos) - min(inf["submit_s"] for inf in infos)
    line = {"mode": "serve", "requests": R, "rate_per_s": args.serve_rate, "steps_per_request": args.serve_steps,
            "stepping": "shared launches (lise_batch)" if args.serve_batching else "separate contexts",
            "precision": "mixed", "hbm_budget_gb": args.serve_budget_gb, "max_active": args.serve_max_active,
            "steps_per_turn": args.serve_turn,
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "mean": float(lat.mean()), "max": float(lat.max())},
            "queue_wait_s": {"p50": float(np.percentile(queue, 50)), "mean": float(queue.mean())},
            "throughput": units / makespan, "unit": UNIT, "makespan_s": makespan,
            "peak_used_gb": st["peak_used_bytes"] / 1e9, "peak_active": st["peak_active"],
            "all_ok": all(inf["status"] == 0 for inf in infos),
            "mix": {"lattices": [int(x) for x in lattices], "n_qp": [int(x) for x in nqps]}}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """A batch of independent evolutions of uneven size through the serving loop.

    --batch-evolutions evolutions (default 64, seed 7): lattice from {16, 24, 32, 40}^3,
    state count uniform in [128, 4096], drive amplitude A uniform in [0, 0.05]
    (Omega 0.3), mixed precision, --batch-steps ABM steps each.  All are ready at
    t = 0; their summed device footprint is far above one GPU's memory, so the
    server admits them as budget frees up (waves), first fit in arrival order
    with at most --batch-max-skips passes over any one evolution.  All are
    submitted at t = 0 without host copies (the server reads each initial state
    from the caller's array at admission).  Reported: aggregate throughput,
    makespan and the schedule.  The active evolutions are stepped together in shared
    launches (lise_batch through the server's batching) unless --batch-separate."""
    import numpy as np
    from paper_2009_00745_b300 import lise as L
    from paper_2009_00745_b300 import workloads as Wl
    rng = np.random.default_rng(7)
    R = args.batch_evolutions
    lattices = rng.choice([16, 24, 32, 40], R)
    nqps = rng.integers(128, 4097, R)
    amps = rng.uniform(0.0, 0.05, R)
    base = {}
    for n in sorted(set(int(x) for x in lattices)):
        q = int(max(nq for nq, l in zip(nqps, lattices) if l == n))
        w = Wl.ufg_plane_waves(n, q, noise_eps=1e-3, precision="mixed", steps=args.batch_steps)
        base[n] = (w, w.initial_state())
    budget = int(args.batch_budget_gb * 1e9)
    fps = [L.footprint_bytes(int(l), int(nq), precision="mixed") for l, nq in zip(lattices, nqps)]
    with L.Server(budget, max_active=args.batch_max_active, steps_per_turn=args.batch_turn) as srv:
        srv.set_admission("first_fit", max_skips=args.batch_max_skips)
        if not args.batch_separate:
            srv.set_batching(True)
        t0 = time.perf_counter()
        ids = []
        for i in range(R):
            w, psi = base[int(lattices[i])]
            nq = int(nqps[i])
            ids.append(srv.submit(w.nx, nq, psi[:nq], 0.0, w.dt, args.batch_steps, a=w.a, alpha=w.alpha,
                                  beta=w.beta, mu=w.mu, g=w.g, drive_A=float(amps[i]), drive_Omega=0.3,
                                  precision="mixed", copy=False))
        infos = [srv.wait(rid, want_state=False)[1] for rid in ids]
        st = srv.stats()
        wall = time.perf_counter() - t0
    units = sum(float(nq) * int(l) ** 3 * args.batch_steps for nq, l in zip(nqps, lattices))
    start = min(inf["submit_s"] for inf in infos)
    makespan = max(inf["done_s"] for inf in infos) - start
    # the admission schedule and, at 20 instants, how many evolutions (and GB) were resident
    events = sorted((inf["admit_s"] - start, inf["done_s"] - start, i) for i, inf in enumerate(infos))
    schedule = [{"i": int(i), "N": int(lattices[i]), "n_qp": int(nqps[i]), "A": round(float(amps[i]), 4),
                 "footprint_gb": round(fps[i] / 1e9, 2), "admit_s": round(a, 3), "done_s": round(d, 3)}
                for a, d, i in events]
    timeline = []
    for k in range(20):
        tk = (k + 0.5) * makespan / 20
        live = [i for a, d, i in events if a <= tk < d]
        timeline.append({"t_s": round(tk, 2), "active": len(live),
                         "resident_gb": round(sum(fps[i] for i in live) / 1e9, 1)})
    line = {"mode": "batch", "evolutions": R, "steps_per_evolution": args.batch_steps, "precision": "mixed",
            "stepping": "separate contexts" if args.batch_separate else "shared launches (lise_batch)",
            "hbm_budget_gb": args.batch_budget_gb, "max_active": args.batch_max_active,
            "admission": "first fit, max %d skips" % args.batch_max_skips,
            "steps_per_turn": args.batch_turn, "sum_footprint_gb": round(sum(fps) / 1e9, 1),
            "throughput": units / makespan, "unit": UNIT, "makespan_s": makespan, "wall_s": wall,
            "peak_used_gb": st["peak_used_bytes"] / 1e9, "peak_active": st["peak_active"],
            "all_ok": all(inf["status"] == 0 for inf in infos),
            "active_timeline": timeline, "schedule": schedule}
    print(json.dumps(line), flush=True)
    return 0


def config_of(w, args):
    return {"workload": w.name, "lattice": f"{w.nx}^3", "n_qp": w.n_qp, "dt": w.dt,
            "precision": w.precision, "steps_in_workload": w.steps,
            "l2": "inputs larger than L2 (state + ABM history %.1f GB, no flush)" % (
                {"fp64": 10 * 16, "mixed": 3 * 16 + 7 * 8, "mixed_strict": 5 * 16 + 5 * 8}[w.precision]
                * w.n_qp * 2 * w.nxyz / 1e9)}


def roofline(w, prof, ms_per_step, fp64_peak):
    """Roofline of the dominant kernel class from the live per-launch event times.

    frac: FP64 path, the fully fused byte model (FUSED_BYTES: 480 B per (state, site,
    step)) attributed to the two pencils launches of a step (the fused step's two kernels),
    per launch, over the mean launch time, against the measured HBM copy bandwidth; mixed
    path (whose step also has a streaming predictor launch), the kernel's own bytes as
    designed.  step: the fused model's bytes (480 or 448 B) over the whole step time.
    design: the kernel's own traffic as designed (algorithmic_per_qp_site), for comparison
    with the ncu traffic.  fp64_pipe (FP64 path): the FP64 flops the pencils kernel
    executes over its launch time, against the measured FP64 FMA peak."""
    mixed = w.precision != "fp64"
    alg = algorithmic_per_qp_site(w.nx, mixed, strict=w.precision == "mixed_strict")
    dom = max((k for k in ("planes", "pencils", "pointwise") if alg[k]["launches_per_step"]),
              key=lambda k: prof[k][1])
    launches, tot_ms = prof[dom]
    per_launch_ms = tot_ms / max(launches, 1)
    qp_sites = float(w.n_qp) * w.nxyz
    hbm_peak, hbm_src = read_peaks()
    a = alg[dom]
    design_bytes = a["bytes"] * qp_sites / a["launches_per_step"]
    fused = FUSED_BYTES[mixed]
    if dom == "pencils" and not mixed:
        # the FP64 pencils launches are the fused step's two kernels (the predictor is in the
        # derivative launch's epilogue); only the in-plane kinetic part runs outside them
        bytes_per_launch = fused * qp_sites / 2
        model = "%d B per (state, site, step) fully fused, over 2 pencils launches per step" % fused
    else:
        # the mixed path splits the step over pencils, a streaming predictor and the in-plane
        # kernel: each kernel against its own bytes as designed; the fused model is `step`
        bytes_per_launch = design_bytes
        model = "the kernel's own bytes as designed (algorithmic_per_qp_site)"
    gbs = bytes_per_launch / (per_launch_ms / 1e3) / 1e9
    step_gbs = fused * qp_sites / (ms_per_step / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak,
            "peak_source": hbm_src + " (MEASURED_PEAKS.json hbm_gbs)", "kernel": dom,
            "traffic": recorded_traffic(w.name, dom, w.precision), "launch_ms": per_launch_ms,
            "algorithmic_bytes_per_launch": bytes_per_launch, "byte_model": model,
            "step": {"achieved": step_gbs, "frac": step_gbs / hbm_peak, "bytes_per_step": fused * qp_sites},
            "design_bytes_per_launch": design_bytes,
            "kernel_share": {k: v[1] / max(sum(x[1] for x in prof.values()), 1e-30) for k, v in prof.items()}}
    if not mixed and dom == "pencils" and fp64_peak:
        tflops = a["flops"] * qp_sites / a["launches_per_step"] / (per_launch_ms / 1e3) / 1e12
        roof["fp64_pipe"] = {"achieved_tflops": tflops, "peak_tflops": fp64_peak, "frac": tflops / fp64_peak,
                             "peak_source": "measured (lise_measure_fp64_peak, FMA chains)",
                             "flops_per_launch": a["flops"] * qp_sites / a["launches_per_step"]}
    return roof


def measure(L, w, psi_dev, args, local, stream, drift_steps=0, drift_every=25, clocks=True, barrier=None):
    """Device throughput of w (CUDA events on the context stream around K profiled steps after
    W warm-up steps), plus, with drift_steps, the energy sampled at fixed step counts of one
    evolution (0, then every drift_every steps up to drift_steps; the timed steps are part of
    it).  Returns a dict; the context is freed."""
    ctx = L.Context.from_workload(w, device=local, stream=stream.cuda_stream)
    ctx.set_state(psi_dev, 0.0, w.dt)
    done, E = 0, []
    sample_at = set(range(0, drift_steps + 1, drift_every)) if drift_steps else set()

    def advance(k):
        nonlocal done
        while k > 0:
            nxt = min([s for s in sample_at if s > done] + [done + k])
            ctx.step(nxt - done)
            k -= nxt - done
            done = nxt
            if done in sample_at:
                E.append((done, ctx.energy()[0]))

    if 0 in sample_at:
        E.append((0, ctx.energy()[0]))
    advance(args.warmup)
    ctx.sync()
    sampler = ClockSampler(local) if clocks else None
    if sampler:
        sampler.start()
        time.sleep(0.4)
    if barrier:
        barrier()
    torch_sync()
    ctx.profile(True)
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed_steps")  # (lets a profiler select exactly these launches)
    e0.record(stream)
    ctx.step(args.steps)
    e1.record(stream)
    e1.synchronize()
    torch.cuda.nvtx.range_pop()
    torch_sync()
    if barrier:
        barrier()
    clk = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1)
    prof = ctx.profile_read()
    ctx.profile(False)
    done += args.steps
    if done in sample_at:
        E.append((done, ctx.energy()[0]))
    if drift_steps > done:
        advance(drift_steps - done)
    E_end, N_end = ctx.energy()
    ctx.close()
    return {"ms": ms, "prof": prof, "clocks": clk, "E": E, "E_end": E_end, "N_end": N_end,
            "units": float(w.n_qp) * w.nxyz * args.steps}


def torch_sync():
    import torch
    torch.cuda.synchronize()


def upload_state(w, local):
    import torch
    psi_host = torch.empty((w.n_qp, 2, w.nz, w.ny, w.nx), dtype=torch.complex128, pin_memory=True)
    w.initial_state(out=psi_host.numpy())
    psi_dev = psi_host.to(f"cuda:{local}")
    torch.cuda.synchronize()
    return psi_host, psi_dev


def run_pair(L, args, local, stream, fp64_peak):
    """The metric's comparison: one workload in both precisions (default: the driven 48^3
    lattice with 4096 states), same K and W, each timed like the headline, and the mixed
    path's energy against the FP64 trajectory over --pair-drift-steps steps."""
    from paper_2009_00745_b300 import workloads as Wl
    import torch
    w = Wl.named(args.pair_workload)
    psi_host, psi_dev = upload_state(w, local)
    del psi_host
    out = {"workload": w.name, "lattice": f"{w.nx}^3", "n_qp": w.n_qp, "steps": args.steps,
           "warmup": args.warmup, "drift_steps": args.pair_drift_steps}
    res = {}
    for prec in ("fp64", "mixed"):
        w.precision = prec
        r = measure(L, w, psi_dev, args, local, stream, drift_steps=args.pair_drift_steps,
                    drift_every=args.pair_drift_every)
        res[prec] = r
        out[prec] = {"value": r["units"] / (r["ms"] / 1e3), "ms_per_step": r["ms"] / args.steps,
                     "roofline": roofline(w, r["prof"], r["ms"] / args.steps, fp64_peak), "clocks": r["clocks"],
                     "gpu_launches": int(sum(v[0] for v in r["prof"].values())),
                     "tuned": {"pencils_states_per_batch": L.pencil_batch(w.nx, prec),
                               "planes_per_block": L.planes_per_block(w.nx, prec)}}
        torch.cuda.empty_cache()
    del psi_dev
    torch.cuda.empty_cache()
    f, m = res["fp64"], res["mixed"]
    ef, em = dict(f["E"]), dict(m["E"])
    common = sorted(set(ef) & set(em))
    dev = max(abs(em[k] - ef[k]) / abs(ef[k]) for k in common) if common else None
    out["mixed_over_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    out["energy_drift"] = {"max_rel_dev_mixed_vs_fp64": dev, "samples_at_steps": common,
                           "criterion": 1e-6, "fp64_energy": [ef[k] for k in common],
                           "note": "energy of a truncated state set is not conserved: the FP64 trajectory is the reference"}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="trap32_vortex_fp64")
    ap.add_argument("--precision", default=None, choices=[None, "fp64", "mixed", "mixed_strict"])
    ap.add_argument("--n-qp", type=int, default=None, help="override the workload's state count")
    ap.add_argument("--impl", default="lise", choices=["lise", "reference"])
    ap.add_argument("--ref-states", type=int, default=32)
    ap.add_argument("--cpu-baseline-states", type=int, default=32)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--pair-workload", default="drive48_mixed",
                    help="workload timed in both precisions for the 'pair' object ('' to skip)")
    ap.add_argument("--pair-drift-steps", type=int, default=100)
    ap.add_argument("--pair-drift-every", type=int, default=25)
    ap.add_argument("--drift", action="store_true",
                    help="compare mixed with FP64 over --steps steps instead of timing")
    ap.add_argument("--drift-every", type=int, default=50)
    ap.add_argument("--serve", action="store_true", help="run a Poisson request stream through the server")
    ap.add_argument("--serve-requests", type=int, default=16)
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-steps", type=int, default=100)
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--serve-max-active", type=int, default=8)
    ap.add_argument("--serve-turn", type=int, default=5)
    ap.add_argument("--serve-batching", action="store_true",
                    help="step the active requests of each lattice size in shared launches (lise_batch); "
                         "default: every request on its own context and stream (measured faster)")
    ap.add_argument("--batch", action="store_true",
                    help="run a batch of uneven evolutions through the server in HBM-budgeted waves")
    ap.add_argument("--batch-evolutions", type=int, default=64)
    ap.add_argument("--batch-steps", type=int, default=500)
    ap.add_argument("--batch-budget-gb", type=float, default=200.0)
    ap.add_argument("--batch-max-active", type=int, default=8)
    ap.add_argument("--batch-max-skips", type=int, default=8)
    ap.add_argument("--batch-turn", type=int, default=8, help="steps per turn of the batched evolutions")
    ap.add_argument("--batch-separate", action="store_true",
                    help="step every evolution on its own (no shared launches)")
    ap.add_argument("--pencil-batch", type=int, default=0,
                    help="force the pencils kernel's states per batch (default: autotuned)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    from paper_2009_00745_b300 import workloads as Wl
    w = Wl.named(args.workload, n_qp=args.n_qp)
    if args.precision:
        w.precision = args.precision
    if args.pencil_batch and args.impl != "reference":
        from paper_2009_00745_b300 import lise as L
        L.set_pencil_batch(w.nx, w.precision, args.pencil_batch)

    if args.impl == "reference":
        return run_reference(args, w)
    if args.drift:
        return run_drift(args, w)
    if args.serve:
        return run_serve(args)
    if args.batch:
        return run_batch(args)

    import torch
    from paper_2009_00745_b300 import lise as L

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    mixed = w.precision != "fp64"
    fp64_peak = L.measure_fp64_peak(local)

    # initial state built on the host, uploaded once (not timed for `value`)
    psi_host, psi_dev = upload_state(w, local)

    # ---- timed region: K steps, device events on the context stream (barriers around it)
    r = measure(L, w, psi_dev, args, local, stream, barrier=dist.barrier if world > 1 else None)
    ms = r["ms"]
    value, ms = whole_job_value(ms, r["units"], world, device=f"cuda:{local}")
    del psi_dev
    torch.cuda.empty_cache()
    roof = roofline(w, r["prof"], ms / args.steps, fp64_peak)
    gpu_launches = int(sum(v[0] for v in r["prof"].values()))

    # ---- e2e through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        out_host = torch.empty(psi_host.shape, dtype=psi_host.dtype, pin_memory=True)
        ctx2 = L.Context.from_workload(w, device=local)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx2.set_state(psi_host.numpy(), 0.0, w.dt)
        ctx2.step(args.steps)
        ctx2.state(out=out_host.numpy())
        E2, N2 = ctx2.energy()
        t_e2e = time.perf_counter() - t0
        ctx2.close()
        state_bytes = 16 * w.n_qp * 2 * w.nxyz
        e2e = {"value": world * r["units"] / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": state_bytes / args.steps, "d2h_bytes_per_step": (state_bytes + 16) / args.steps,
               "includes": "set_state from pinned host (H2D + 3 series-expansion start steps), K ABM steps, "
                           "get_state to pinned host, energy"}
        del out_host
    del psi_host

    # ---- the same comparison the metric names: one workload in both precisions
    pair = None
    if args.pair_workload and rank == 0 and world == 1:
        pair = run_pair(L, args, local, stream, fp64_peak)

    # ---- CPU baseline: the oracle on a bounded sample of the same workload
    cpu = None
    if rank == 0 and args.cpu_baseline_states > 0:
        ns = args.cpu_baseline_states
        rate, secs, thr = oracle_sample_rate(w, ns, 2, 0)
        cpu = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle",
               "sample": f"first {ns} of {w.n_qp} states of {w.name}, 2 timed ABM steps after the untimed start"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if not mixed else "f64+c64",
            "data": "synthetic", "config": config_of(w, args), "roofline": roof, "cpu_baseline": cpu,
            "tuned": {"pencils_states_per_batch": L.pencil_batch(w.nx, w.precision),
                      "planes_per_block": L.planes_per_block(w.nx, w.precision)},
            "e2e": e2e, "clocks": r["clocks"], "gpu_launches": gpu_launches,
            "energy_after_timed_steps": r["E_end"], "particle_number": r["N_end"],
            "fp64_fma_peak_tflops": fp64_peak, "pair": pair,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
