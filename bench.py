#!/usr/bin/env python
"""Benchmark of the data-parallel fine propagator and of Parareal on one GB300.

Default workload (one "step" = one call of the C ABI's fine propagator):
one IMEX RK443 fine step of all 256 time slices of the large Galloway-Proctor problem
(1024 x 1024 grid, kz = 0.57, Rm = 1e4, T = 2 pi * 32 split into 256 slices of 786 steps,
slice i starting at t = i T / 256), complex64 fields [256][3][1024][1024] resident in HBM,
through kd_fine_batched: pack to the 2/3 set, the prologue, 4 x (column, row) kernels,
unpack.

value  = 3 n^2 x 256 degrees of freedom x 1 step / device time of the call (Mdof.steps/s),
         summed over ranks (each rank advances its own 256 slices: weak scaling).
e2e    = the same with the fields read from pinned host memory and the result written
         back to pinned host memory inside the timed region.
roofline = the dominant fine kernel (column or row) of the call: its algorithmic bytes
         per launch (two-pass model, complex64) over its average launch time, measured
         with CUDA events on the context stream, against the measured HBM copy peak.
Also reported beside the line: one Parareal solve of the 128^2 Galloway-Proctor problem
(64 slices, time-to-1e-6 against serial fine stepping with the same kernels, k_con,
errors against the complex64 and the complex128 serial fine solutions), clocks during the
timed region, and the CPU FP64 oracle timed on a bounded sample (cpu_baseline).

--config parareal prints the 128^2 Parareal solve as the line (the earlier headline);
--config large runs one Parareal solve of the 1024^2 problem (minutes); --config sweep,
learned, steppers, coarse-sweep, coarse-sweep-roberts run the studies of the other
configurations; --config profile runs small repeatable cases for ncu.

--impl reference times the CPU FP64 oracle (the slow reference program of this
repository) on the host cores, one field per core, on a bounded sample of the same
workload: one fine step of a 1024^2 field per core per step.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WL = {
    "workload": "gp_cp_128x128_parareal_64_slices",
    "flow": "galloway-proctor", "n": 128, "kz": 0.57, "Rm": 100.0, "dt_fine_max": 5e-3,
    "T": 2 * math.pi * 8, "slices": 64, "n_coarse": 128, "dt_coarse_max": 2.0 / 128, "tol": 1e-6,
    "k_max": 64, "prec_fine": "complex64", "prec_coarse": "complex64", "update": "float64",
    "fine_form": "increment",
}
METRIC = "Parareal time-to-1e-6 vs serial fine (1 GB300); fine Mdof·steps/s, HBM % peak"
UNIT = "Mdof*steps/s"
L2_FLUSH_BYTES = 512 << 20

# The default line: one fine step of every slice of the large Galloway-Proctor problem.
FINE_WL = {
    "workload": "gp_cp_1024x1024_fine_step_256_slices",
    "flow": "galloway-proctor", "n": 1024, "kz": 0.57, "Rm": 1e4, "T": 2 * math.pi * 32, "slices": 256,
    "fine_steps_per_slice": 786, "steps_per_call": 1, "prec_fine": "complex64",
    "inputs": "8 seeded |k|^-2 divergence-free fields (seeds 1000 + 8 rank ..) tiled over the 256 slices; "
              "slice i starts at t = i T / 256",
}


def fine_wl_dt():
    return FINE_WL["T"] / FINE_WL["slices"] / FINE_WL["fine_steps_per_slice"]


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def fine_steps_per_slice():
    dT = WL["T"] / WL["slices"]
    return math.ceil(dT / WL["dt_fine_max"] - 1e-9)


def units_per_solve():
    """degrees of freedom x steps of the serial fine solution the solve reproduces"""
    return 3 * WL["n"] ** 2 * WL["slices"] * fine_steps_per_slice()


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(nsteps):
    """Time the oracle's fine propagator for `nsteps` steps of one slice of the workload."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import numpy as np
    import kd_inputs
    from oracle import kd_oracle as O
    n = WL["n"]
    prob = O.Problem(O.GALLOWAY_PROCTOR, n, WL["kz"], WL["Rm"])
    b = kd_inputs.initial_field(n, WL["kz"], 0)
    dT = WL["T"] / WL["slices"]
    S = fine_steps_per_slice()
    t = time.perf_counter()
    O.propagate(b, prob, 0.0, dT / S, nsteps)
    el = time.perf_counter() - t
    return 3 * n * n * nsteps / el / 1e6, el


_BARRIER = None


def _oracle_worker_init(barrier):
    global _BARRIER
    _BARRIER = barrier
    import kd_inputs  # noqa: F401  (imports before the timed region)
    from oracle import kd_oracle  # noqa: F401


def _oracle_slice(task):
    """Pool worker: the oracle's fine propagator over `nsteps` steps of slice i of the
    workload, started together with the other workers; returns its compute time."""
    i, nsteps = task
    import kd_inputs
    from oracle import kd_oracle as O
    n = WL["n"]
    prob = O.Problem(O.GALLOWAY_PROCTOR, n, WL["kz"], WL["Rm"])
    b = kd_inputs.initial_field(n, WL["kz"], i)
    dT = WL["T"] / WL["slices"]
    S = fine_steps_per_slice()
    _BARRIER.wait(timeout=120)
    t = time.perf_counter()
    O.propagate(b, prob, i * dT, dT / S, nsteps)
    return time.perf_counter() - t


def oracle_all_cores(nsteps, repeats=1):
    """The oracle's fine phase with one slice per host core, as in the paper's layout of
    one time slice per core: a spawn pool of single-threaded workers that start each round
    together.  Returns (cores, [time of the slowest worker, per round])."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    cores = max(1, min(cores, WL["slices"]))
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores)
    pool = ctx.Pool(cores, initializer=_oracle_worker_init, initargs=(barrier,))
    try:
        worst = [max(pool.map_async(_oracle_slice, [(i, nsteps) for i in range(cores)], chunksize=1).get(600))
                 for _ in range(repeats)]
    finally:
        pool.terminate()
        pool.join()
    return cores, worst


def oracle_sample_all_cores(nsteps):
    """One round of oracle_all_cores as a cpu_baseline-style record (Mdof.steps/s over the
    slowest worker's time)."""
    cores, worst = oracle_all_cores(nsteps)
    return {"value": 3 * WL["n"] ** 2 * nsteps * cores / worst[0] / 1e6, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": "%d RK443 fine steps of each of %d slices of the 128^2 GP problem, one slice per core "
                      "(spawned single-threaded workers started together), numpy FP64 oracle, %.1f s"
                      % (nsteps, cores, worst[0])}


def oracle_extrapolated(n, kz, Rm, dt, S, N, nsteps):
    """The oracle's fine propagator timed for `nsteps` steps of one GP slice of an n^2
    workload whose full CPU run is out of reach, and the serial fine run of S steps x N
    slices that this time per step implies (reported as extrapolated)."""
    import kd_inputs
    from oracle import kd_oracle as O
    prob = O.Problem(O.GALLOWAY_PROCTOR, n, kz, Rm)
    b = kd_inputs.initial_field(n, kz, 0)
    O.propagate(b, prob, 0.0, dt, 1)
    t = time.perf_counter()
    O.propagate(b, prob, 0.0, dt, nsteps)
    per = (time.perf_counter() - t) / nsteps
    return {"value": 3 * n * n / per / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle", "extrapolated": True,
            "sample": "%d RK443 fine steps of one %d^2 GP slice, numpy FP64 oracle, %.3f s per step" % (nsteps, n, per),
            "serial_fine_s_extrapolated": per * S * N}


def _oracle_field_step(task):
    """Pool worker: one oracle fine step of the 1024^2 field of slice i of the default
    workload, started together with the other workers; returns its compute time."""
    i, nsteps = task
    import kd_inputs
    from oracle import kd_oracle as O
    W = FINE_WL
    prob = O.Problem(O.GALLOWAY_PROCTOR, W["n"], W["kz"], W["Rm"])
    b = kd_inputs.initial_field(W["n"], W["kz"], 1000 + i % 8)
    _BARRIER.wait(timeout=300)
    t = time.perf_counter()
    O.propagate(b, prob, i * W["T"] / W["slices"], fine_wl_dt(), nsteps)
    return time.perf_counter() - t


def run_reference(args):
    """The CPU FP64 oracle on the default workload: every host core advances one 1024^2
    slice by one fine step per reference step (spawned single-threaded workers started
    together; the step time is the slowest worker's)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import multiprocessing as mp
    W = FINE_WL
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    cores = max(1, min(cores, W["slices"]))
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(cores)
    pool = ctx.Pool(cores, initializer=_oracle_worker_init, initargs=(barrier,))
    try:
        secs = [max(pool.map_async(_oracle_field_step, [(i, 1) for i in range(cores)], chunksize=1).get(900))
                for _ in range(args.warmup + args.steps)][args.warmup:]
    finally:
        pool.terminate()
        pool.join()
    units = 3 * W["n"] ** 2 * cores
    value = args.steps * units / sum(secs) / 1e6
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(FINE_WL),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "one RK443 fine step of one 1024^2 GP slice per core per step, %d cores, "
                                   "numpy FP64 oracle" % cores},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            v = [x.strip() for x in line.split(",")]
            if len(v) < 9:
                continue
            try:
                sm.append(float(v[1]))
                smax.append(float(v[2]))
            except ValueError:
                continue
            for nm, flag in zip(names, v[5:9]):
                if flag.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- roofline
def col_row_bytes(n, batch_slices):
    """Algorithmic bytes of one column launch and of one row launch (complex64):
    the column pass reads and writes the mixed field (3 x P x n); the row pass reads
    and writes it too and touches 3.5 compact spectral arrays (3 x P x P) on average
    over the four stages (stage reads + writes: 4, 5, 3, 2)."""
    K = n // 3
    P = 2 * K + 1
    mixed = 3 * P * n * 8
    spec = 3 * P * P * 8
    return 2 * mixed * batch_slices, (2 * mixed + 3.5 * spec) * batch_slices


# --------------------------------------------------- learned coarse propagator run
LEARNED_WL = {
    "workload": "gp_cp_256x256_parareal_128_slices_learned_coarse",
    "flow": "galloway-proctor", "n": 256, "kz": 0.57, "Rm": 1000.0, "slices": 128, "slice": 2 * math.pi / 16,
    "fine_steps_per_slice": 800, "coarse_dt_over_fine_dt": 20, "learned_modes": 49, "phases": 16,
    "pairs_per_phase": 256, "epochs": 300, "lr": 0.5, "optimizer": "minnorm (closed form) and momentum",
    "tol": 1e-6, "k_max": 32,
    "pair_count_study": {"phases": [0, 1], "pairs": [64, 256, 1024], "heldout_per_phase": 64},
}


def run_learned(args):
    """Time-to-solution of Parareal with the learned coarse propagator against the
    classical coarse propagator (20x the fine step, same mode set) and serial fine
    stepping, GP 256^2, Rm = 1000, 128 slices of 2 pi / 16."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import kd_inputs
    import paper_1902_00387_gb300 as kd
    from oracle import kd_oracle as O
    kd.load()
    torch.cuda.init()
    W = LEARNED_WL
    n, N, m = W["n"], W["slices"], W["learned_modes"]
    T = N * W["slice"]
    dt = W["slice"] / W["fine_steps_per_slice"]
    dtc = dt * W["coarse_dt_over_fine_dt"]
    b0 = torch.tensor(kd_inputs.initial_field(n, W["kz"], 1000)).cuda()
    out = {"impl": "ours", "config": dict(W), "metric": "Parareal time-to-1e-6, learned vs classical coarse",
           "unit": "ms", "higher_is_better": False}

    def ctx_for(kind):
        p = kd.make_params(kd.KD_FLOW_GALLOWAY_PROCTOR, n, W["kz"], W["Rm"], dt, kd.KD_C64, n_coarse=64,
                           dt_coarse=dtc, prec_coarse=kd.KD_C64, fine_form=kd.KD_FINE_INCREMENT, learned_modes=m,
                           coarse_kind=kind)
        return kd.kd_create(p)

    def solve(ctx):
        u = torch.zeros((N + 1, 3, n, n), dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s, st = kd.kd_parareal_run(ctx, b0, T, N, W["k_max"], W["tol"], u)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), st, u

    # classical coarse propagator on the same mode set
    ctx = ctx_for(kd.KD_COARSE_CLASSICAL)
    solve(ctx)
    ms_c, st_c, u_c = solve(ctx)
    ser = torch.zeros_like(u_c)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    kd.kd_fine_serial(ctx, b0, T, N, ser)
    e1.record()
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1)
    kd.kd_destroy(ctx)

    # the classical propagator with the fine step on the same set (20x the work of the
    # benched one): how much accuracy of G on the set alone buys in iterations
    p1 = kd.make_params(kd.KD_FLOW_GALLOWAY_PROCTOR, n, W["kz"], W["Rm"], dt, kd.KD_C64, n_coarse=64,
                        dt_coarse=dt, prec_coarse=kd.KD_C64, fine_form=kd.KD_FINE_INCREMENT, learned_modes=m,
                        coarse_kind=kd.KD_COARSE_CLASSICAL)
    ctx = kd.kd_create(p1)
    ms_a, st_a, u_a = solve(ctx)
    acc = {"ms": ms_a, "k_con": st_a.k_con, "converged": bool(st_a.converged),
           "sigma": list(st_a.sigma[:st_a.k_con])}
    kd.kd_learned_init(ctx, W["phases"], W["slice"])
    acc_ctx = ctx

    # learned: build from the classical propagator, pairs from the fine propagator, train
    ctx = ctx_for(kd.KD_COARSE_LEARNED)
    t = time.perf_counter()
    kd.kd_learned_init(ctx, W["phases"], W["slice"])
    t_init = time.perf_counter() - t

    def inputs(seed0, count):
        # seeded |k|^-2 fields drawn on an 80^2 grid (|k| <= 26 covers the set)
        x = np.stack([O.learned_restrict(kd_inputs.initial_field(80, W["kz"], seed0 + i), m) for i in range(count)])
        return torch.tensor(x.astype(np.complex64), device="cuda")

    def pairs(xt, ph):
        yt = torch.zeros_like(xt)
        kd.kd_learned_pairs(ctx, xt, len(ph), ph, yt)
        return yt

    npair = W["pairs_per_phase"] * W["phases"]
    t = time.perf_counter()
    xt = inputs(10_000, npair)
    ph = np.arange(npair) % W["phases"]
    yt = pairs(xt, ph)
    t_pairs = time.perf_counter() - t
    nv = 16 * W["phases"]
    xvt = inputs(90_000, nv)
    phv = np.arange(nv) % W["phases"]
    yvt = pairs(xvt, phv)
    # the classical operator as stored (BF16 matrix) before any training
    e_bf16, ec = kd.kd_learned_eval(ctx, xvt, yvt, phv, nv, W["phases"])
    _, e_acc = kd.kd_learned_eval(acc_ctx, xvt, yvt, phv, nv, W["phases"])
    acc["heldout_err_median"] = float(np.median(e_acc))
    kd.kd_destroy(acc_ctx)
    # momentum descent from the classical matrix (the earlier training)
    t = time.perf_counter()
    loss = kd.kd_learned_train(ctx, xt, yt, ph, npair, W["epochs"], W["lr"], 0.0, W["phases"], kd.KD_TRAIN_MOMENTUM)
    t_mom = time.perf_counter() - t
    e_mom, _ = kd.kd_learned_eval(ctx, xvt, yvt, phv, nv, W["phases"])
    # The closed-form minimiser (KD_TRAIN_MINNORM; what momentum descent tends to) on the
    # study phases: its ridge lambda = alpha mean |x|^2 chosen on held-out pairs, then the
    # held-out error against the number of pairs.
    PS = W["pair_count_study"]
    mmax, nh = max(PS["pairs"]), PS["heldout_per_phase"]
    phs = np.array(PS["phases"] * mmax)
    xs = inputs(200_000, len(phs))
    ys = pairs(xs, phs)
    phh = np.array(PS["phases"] * nh)
    xh = inputs(300_000, len(phh))
    yh = pairs(xh, phh)
    msq = float((torch.linalg.norm(xs.reshape(len(phs), -1), dim=1) ** 2).mean())

    def minnorm(x_, y_, ph_, alpha, mm):
        kd.kd_learned_train(ctx, x_, y_, ph_, len(ph_), 0, 0.0, alpha * msq / mm, W["phases"], kd.KD_TRAIN_MINNORM)

    def study_err(mm, alpha):
        k = mm * len(PS["phases"])
        minnorm(xs[:k], ys[:k], phs[:k], alpha, mm)
        a, c = kd.kd_learned_eval(ctx, xh, yh, phh, len(phh), W["phases"])
        return [float(a[p]) for p in PS["phases"]], [float(c[p]) for p in PS["phases"]]

    alphas = [0.0, 1e-4, 1e-3, 1e-2, 1e-1]
    m0 = W["pairs_per_phase"]
    by_alpha = []
    for a_ in alphas:
        e_, c_ = study_err(m0, a_)
        by_alpha.append({"alpha": a_, "heldout_err": e_, "heldout_err_classical": c_})
    best = min(by_alpha, key=lambda r: float(np.mean(r["heldout_err"])))["alpha"]
    curve = []
    for mm in PS["pairs"]:
        for a_ in sorted({0.0, best}):
            e_, c_ = study_err(mm, a_)
            curve.append({"pairs_per_phase": mm, "alpha": a_, "heldout_err_minnorm": e_, "heldout_err_classical": c_})
    # every phase with the chosen ridge, then the solve
    t = time.perf_counter()
    minnorm(xt, yt, ph, best, W["pairs_per_phase"])
    torch.cuda.synchronize()
    t_mn = time.perf_counter() - t
    el, ec = kd.kd_learned_eval(ctx, xvt, yvt, phv, nv, W["phases"])
    solve(ctx)
    ms_l, st_l, u_l = solve(ctx)
    kd.kd_destroy(ctx)
    err = lambda u: (torch.linalg.norm(u[-1] - ser[-1]) / torch.linalg.norm(ser[-1])).item()
    # What no operator on the set can change: Parareal's update leaves the modes outside the
    # set to the fine propagator alone (the coarse propagator is zero there), so their error
    # after iteration k + 1 is P F applied to the error of iteration k.  Its outside-to-outside
    # block P F P over one slice (from t = 0) is measured by power iteration; its norm bounds
    # the per-iteration contraction of that part of the defect for any coarse operator.
    fctx = kd.kd_create(kd.make_params(kd.KD_FLOW_GALLOWAY_PROCTOR, n, W["kz"], W["Rm"], dt, kd.KD_C128))
    kk = torch.fft.fftfreq(n, 1.0 / n, device="cuda").round().long()
    inside = ((kk[None, :] >= -(m // 2)) & (kk[None, :] < m - m // 2) &
              (kk[:, None] >= -(m // 2)) & (kk[:, None] < m - m // 2))
    v = torch.tensor(kd_inputs.initial_field(n, W["kz"], 4242), device="cuda")
    v[:, inside] = 0
    v /= torch.linalg.norm(v)
    t00 = torch.zeros(1, dtype=torch.float64, device="cuda")
    rho_hist = []
    w = torch.empty_like(v)
    for _ in range(30):
        kd.kd_fine_batched(fctx, v[None], w[None], t00, W["fine_steps_per_slice"], 1, kd.KD_C128)
        w[:, inside] = 0
        r = torch.linalg.norm(w).item()
        rho_hist.append(r)
        v = w / r
    kd.kd_destroy(fctx)
    outside_frac = (torch.linalg.norm(ser[-1][:, ~inside]) / torch.linalg.norm(ser[-1])).item()
    sc = list(st_c.sigma[:st_c.k_con])
    out.update({
        "serial_fine_ms": ms_s,
        "classical": {"ms": ms_c, "k_con": st_c.k_con, "sigma": sc, "converged": bool(st_c.converged),
                      "err_vs_serial_fine": err(u_c), "speedup_vs_serial_fine": ms_s / ms_c,
                      "growth_rate": st_c.growth_rate,
                      "sigma_ratio_last8": [sc[i + 1] / sc[i] for i in range(max(0, len(sc) - 9), len(sc) - 1)]},
        "learned": {"ms": ms_l, "k_con": st_l.k_con, "sigma": list(st_l.sigma[:st_l.k_con]),
                    "converged": bool(st_l.converged), "method": "minnorm", "ridge_alpha": best,
                    "fallback_used": bool(st_l.fallback_used), "err_vs_serial_fine": err(u_l),
                    "speedup_vs_serial_fine": ms_s / ms_l, "phases_kept": int(np.sum(el <= ec)),
                    "heldout_err_minnorm_median": float(np.median(el)),
                    "heldout_err_momentum_median": float(np.median(e_mom)),
                    "heldout_err_classical_bf16_median": float(np.median(e_bf16)),
                    "heldout_err_classical_median": float(np.median(ec)),
                    "train_loss_momentum_first_last": [float(loss[:, 0].mean()), float(loss[:, -1].mean())],
                    "init_s": t_init, "pairs_s": t_pairs, "train_momentum_s": t_mom, "train_minnorm_s": t_mn},
        "classical_fine_step_on_set": acc,
        "ridge_study": by_alpha,
        "pair_count_study": curve,
        "outside_set": {"modes": "kx, ky outside [-%d, %d)" % (m // 2, m - m // 2),
                        "norm_fraction_of_serial_fine_final_state": outside_frac,
                        "rho_outside_block_one_slice": rho_hist[-1], "rho_history": rho_hist},
    })
    out["value"] = ms_l
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_extrapolated(n, W["kz"], W["Rm"], dt, W["fine_steps_per_slice"], N, 4)
    print(json.dumps(out), flush=True)


# ------------------------------------------------- stepper work versus accuracy (Sec. 5.1)
STEPPERS_WL = {
    "workload": "gp_cp_128x128_stepper_work_vs_accuracy", "flow": "galloway-proctor", "n": 128, "kz": 0.57,
    "Rm": 100.0, "T": 2 * math.pi / 8, "batch": 64, "reference": "RK443, dt = T/4096, complex128",
    "dts": [0.04, 0.02, 0.01, 0.005, 0.0025, 0.00125],
}


def run_steppers(args):
    """The paper's stepper study (Sec. 5.1): relative error at T of RK111, RK222 and RK443
    against a reference run, and the device time of the batched FP32 fine propagation
    (64 fields), per step size."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import kd_inputs
    import paper_1902_00387_gb300 as kd
    kd.load()
    torch.cuda.init()
    W = STEPPERS_WL
    n, T, B = W["n"], W["T"], W["batch"]
    b = kd_inputs.initial_batch(n, W["kz"], range(B))
    t0 = torch.zeros(B, dtype=torch.float64, device="cuda")

    def run(sch, dt_max, prec):
        steps = math.ceil(T / dt_max - 1e-9)     # equal steps that end exactly at T
        ctx = kd.kd_create(kd.make_params(kd.KD_FLOW_GALLOWAY_PROCTOR, n, W["kz"], W["Rm"], T / steps, prec,
                                          fine_scheme=sch))
        try:
            dtype = torch.complex64 if prec == kd.KD_C64 else torch.complex128
            x = torch.tensor(b, dtype=dtype, device="cuda")
            y = torch.empty_like(x)
            kd.kd_fine_batched(ctx, x, y, t0, steps, B, prec)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            kd.kd_fine_batched(ctx, x, y, t0, steps, B, prec)
            e1.record()
            torch.cuda.synchronize()
            return y.to(torch.complex128), e0.elapsed_time(e1), steps
        finally:
            kd.kd_destroy(ctx)

    ref, _, _ = run(kd.KD_RK443, T / 4096, kd.KD_C128)
    rows = []
    for name, sch, stages in (("RK111", kd.KD_RK111, 1), ("RK222", kd.KD_RK222, 2), ("RK443", kd.KD_RK443, 4)):
        for dt in W["dts"]:
            y, ms, steps = run(sch, dt, kd.KD_C64)
            err = (torch.linalg.norm(y - ref) / torch.linalg.norm(ref)).item()
            rows.append({"scheme": name, "dt": T / steps, "steps": steps, "rhs_evals": steps * stages,
                         "rel_error": err if math.isfinite(err) else None, "ms": ms})
    print(json.dumps({"config": W, "metric": "relative error at T vs device time (64 fields, complex64)",
                      "rows": rows}), flush=True)


# --------------------------------------------------------- coarse-grid sweep (Sec. 5.2)
def run_coarse_sweep(args):
    """The paper's coarse-resolution study (Sec. 5.2, fig. 6) on the GP 128^2, 64-slice problem of the headline:
    Parareal iterations and time to 1e-6 for N_C = 16, 32, 64, 128 (coarse step at the
    stability limit of each coarse grid, min(20 dt, 2 / N_C): explicit RK443 on an N_C grid
    blows up above ~2.5 / N_C to 3 / N_C), against the serial fine time with the same
    kernels."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import kd_inputs
    import paper_1902_00387_gb300 as kd
    kd.load()
    torch.cuda.init()
    n, N, T = WL["n"], WL["slices"], WL["T"]
    b0 = torch.tensor(kd_inputs.initial_field(n, WL["kz"], 1000), device="cuda")
    rows = []
    serial = None
    for nc in (16, 32, 64, 128):
        dtc = min(20 * WL["dt_fine_max"], 2.0 / nc)
        p = kd.make_params(kd.KD_FLOW_GALLOWAY_PROCTOR, n, WL["kz"], WL["Rm"], WL["dt_fine_max"], kd.KD_C64,
                           n_coarse=nc, dt_coarse=dtc, prec_coarse=kd.KD_C64, fine_form=kd.KD_FINE_INCREMENT)
        ctx = kd.kd_create(p)
        try:
            kd.kd_autotune(ctx, kd.KD_GRID_FINE, N, 2)
            if serial is None:
                ser = torch.zeros((N + 1, 3, n, n), dtype=torch.complex128, device="cuda")
                kd.kd_fine_serial(ctx, b0, T, N, ser)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                kd.kd_fine_serial(ctx, b0, T, N, ser)
                e1.record()
                torch.cuda.synchronize()
                serial = e0.elapsed_time(e1)
            kd.kd_parareal_run(ctx, b0, T, N, WL["k_max"], WL["tol"])
            ms = []
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                s, st = kd.kd_parareal_run(ctx, b0, T, N, WL["k_max"], WL["tol"])
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            rows.append({"n_coarse": nc, "dt_coarse": st.dt_coarse_used, "coarse_steps": st.n_coarse_steps,
                         "k_con": st.k_con, "converged": bool(st.converged), "ms": min(ms),
                         "fine_ms": st.ms_fine, "coarse_ms": st.ms_coarse, "speedup_vs_serial_fine": serial / min(ms)})
        finally:
            kd.kd_destroy(ctx)
    print(json.dumps({"config": dict(WL, study="n_coarse sweep"), "serial_fine_ms": serial, "rows": rows}),
          flush=True)


# ------------------------------------------- coarse-resolution study, Roberts (Sec. 5.2)
ROBERTS_SWEEP_WL = {
    "workload": "roberts_rm512_nf160_parareal_10_slices_nc_sweep",
    "flow": "roberts", "n": 160, "kz": 2.87, "Rm": 512.0, "dt_fine": 1e-2, "T": 50.0, "slices": 10,
    "n_coarse": [20, 40, 60, 80, 100, 120, 160], "dt_coarse": "dt_fine * N_F / N_C (the stability limit ~1.6 / N)",
    "tol": 1e-6, "k_max": 10, "prec_fine": "complex64", "prec_coarse": "complex64", "update": "float64",
    "fine_form": "increment",
}


def run_roberts_coarse_sweep(args):
    """The paper's coarse-resolution study at its own parameters (Sec. 5.2, fig. 6 and
    Table 1's Roberts row): Rm = 512, kz = 2.87, N_F = 160, delta t = 1e-2, N_P = 10
    slices, the coarse step at the stability limit of each coarse grid; Parareal
    iterations and time to the tolerance against the serial fine run, one GPU."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import kd_inputs
    import paper_1902_00387_gb300 as kd
    kd.load()
    torch.cuda.init()
    W = dict(ROBERTS_SWEEP_WL, fine_operator=args.fine_operator + (" (mixed-radix 5 x 32 FFT)" if args.fine_operator
                                                                    == "fft" else " (spectral convolution)"))
    fine_op = kd.KD_FINE_CONV if args.fine_operator == "conv" else kd.KD_FINE_FFT
    n, N, T = W["n"], W["slices"], W["T"]
    b0 = torch.tensor(kd_inputs.initial_field(n, W["kz"], 1000), device="cuda")

    def timed(f, reps=3):
        f()
        best = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = f()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best, out

    rows, serial = [], None
    for nc in W["n_coarse"]:
        dtc = W["dt_fine"] * n / nc
        p = kd.make_params(kd.KD_FLOW_ROBERTS, n, W["kz"], W["Rm"], W["dt_fine"], kd.KD_C64, n_coarse=nc,
                           dt_coarse=dtc, prec_coarse=kd.KD_C64, fine_form=kd.KD_FINE_INCREMENT,
                           fine_operator=fine_op)
        ctx = kd.kd_create(p)
        try:
            if serial is None:
                ser = torch.zeros((N + 1, 3, n, n), dtype=torch.complex128, device="cuda")
                serial, _ = timed(lambda: kd.kd_fine_serial(ctx, b0, T, N, ser))
                ser_last = ser[-1].clone()
            out = torch.zeros((N + 1, 3, n, n), dtype=torch.complex128, device="cuda")
            ms, (s, st) = timed(lambda: kd.kd_parareal_run(ctx, b0, T, N, W["k_max"], W["tol"], out))
            err = float(torch.linalg.vector_norm(out[-1] - ser_last) / torch.linalg.vector_norm(ser_last))
            rows.append({"n_coarse": nc, "dt_coarse": st.dt_coarse_used, "coarse_steps": st.n_coarse_steps,
                         "k_con": st.k_con, "converged": bool(st.converged), "ms": ms, "fine_ms": st.ms_fine,
                         "coarse_ms": st.ms_coarse, "speedup_vs_serial_fine": serial / ms,
                         "err_vs_serial_fine": err,
                         "sigma": [float(st.sigma[i]) for i in range(min(st.k_con, W["k_max"]))]})
        finally:
            kd.kd_destroy(ctx)
    print(json.dumps({"config": dict(W, study="n_coarse sweep"), "serial_fine_ms": serial, "rows": rows}),
          flush=True)


# ------------------------------------------------- large run (GP 1024^2, 256 slices)
LARGE_WL = {
    "workload": "gp_cp_1024x1024_parareal_256_slices",
    "flow": "galloway-proctor", "n": 1024, "kz": 0.57, "Rm": 1e4, "dt_fine_max": 1e-3, "T": 2 * math.pi * 32,
    "slices": 256, "n_coarse": 512, "tol": 1e-6, "k_max": 32, "prec_fine": "complex64", "prec_coarse": "complex64",
    "update": "float64", "fine_form": "increment", "coarse": "classical (the learned operator is not trained here)",
}


def run_large(args):
    """One Parareal solve of the GP 1024^2 problem with 256 slices resident on
    one GPU, against serial fine stepping with the same kernels; growth rate from the
    log-energy fit; fine-kernel roofline from a separately timed batched step."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import kd_inputs
    import paper_1902_00387_gb300 as kd
    kd.load()
    torch.cuda.init()
    W = LARGE_WL
    n, N, T = W["n"], W["slices"], W["T"]
    dtc = min(20 * W["dt_fine_max"], 2.0 / W["n_coarse"])     # explicit limit ~2.5 / N_C of the coarse grid
    p = kd.make_params(kd.KD_FLOW_GALLOWAY_PROCTOR, n, W["kz"], W["Rm"], W["dt_fine_max"], kd.KD_C64,
                       n_coarse=W["n_coarse"], dt_coarse=dtc, prec_coarse=kd.KD_C64, fine_form=kd.KD_FINE_INCREMENT)
    ctx = kd.kd_create(p)
    kd.kd_autotune(ctx, kd.KD_GRID_FINE, N, 2, os.path.join(tempfile.gettempdir(), "kd_tune_cache.json"))
    kd.kd_autotune(ctx, kd.KD_GRID_COARSE, 1, 4, os.path.join(tempfile.gettempdir(), "kd_tune_cache.json"))
    plan_f, plan_c = kd.kd_get_plan(ctx, kd.KD_GRID_FINE), kd.kd_get_plan(ctx, kd.KD_GRID_COARSE)
    b0 = torch.tensor(kd_inputs.initial_field(n, W["kz"], 1000), device="cuda")
    u = torch.zeros((N + 1, 3, n, n), dtype=torch.complex128, device="cuda")
    ev = lambda: torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(0)
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = ev(), ev()
    e0.record()
    s, st = kd.kd_parareal_run(ctx, b0, T, N, W["k_max"], W["tol"], u)
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    S = st.n_fine_steps
    ser = torch.zeros_like(u)
    e0, e1 = ev(), ev()
    e0.record()
    kd.kd_fine_serial(ctx, b0, T, N, ser)
    e1.record()
    torch.cuda.synchronize()
    ms_ser = e0.elapsed_time(e1)
    err = (torch.linalg.norm(u[-1] - ser[-1]) / torch.linalg.norm(ser[-1])).item()
    gr_ser = kd.kd_growth_rate(ctx, ser, N + 1, T, 0.5 * T)
    del ser, u
    torch.cuda.empty_cache()
    # fine-kernel roofline: two steps of all 256 slices, every launch timed with events
    x = torch.tensor(kd_inputs.initial_batch(n, W["kz"], range(8)), dtype=torch.complex64, device="cuda")
    x = x.repeat(N // 8, 1, 1, 1)
    t0 = torch.arange(N, dtype=torch.float64, device="cuda") * (T / N)
    kd.kd_fine_batched(ctx, x, x, t0, 1, N)
    kd.kd_profile(ctx, 1)
    kd.kd_fine_batched(ctx, x, x, t0, 2, N)
    prof_ms, prof_n = kd.kd_profile_read(ctx)
    kd.kd_profile(ctx, 0)
    cb, rb = col_row_bytes(n, N)
    step_bytes = 4 * (cb + rb)
    achieved = (cb * prof_n[0] + rb * prof_n[1]) / ((prof_ms[0] + prof_ms[1]) / 1e3) / 1e9
    kid = 0 if prof_ms[0] >= prof_ms[1] else 1
    k_ach = ((cb, rb)[kid] * prof_n[kid]) / (prof_ms[kid] / 1e3) / 1e9
    hbm_peak, peak_kind = peaks()
    units = 3 * n * n * N * S
    out = {
        "metric": METRIC, "value": units / (ms / 1e3) / 1e6, "unit": UNIT, "n_gpus": 1, "steps": 1, "warmup": 0,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 fine / f64 update", "data": "synthetic",
        "config": dict(W, dt_coarse=dtc, fine_steps_per_slice=S, coarse_steps_per_slice=st.n_coarse_steps,
                       fine_plan=list(plan_f), coarse_plan=list(plan_c)),
        "time_to_solution_ms": ms, "serial_fine_ms": ms_ser, "speedup_vs_serial_fine": ms_ser / ms,
        "k_con": st.k_con, "converged": bool(st.converged), "sigma": list(st.sigma[:st.k_con]),
        "err_vs_serial_fine": err, "growth_rate": st.growth_rate, "growth_rate_serial_fine": gr_ser,
        "phase_ms": {"fine": st.ms_fine, "coarse_and_update": st.ms_coarse},
        "fine_step": {"ms_per_step_all_slices": (prof_ms[0] + prof_ms[1]) / 2, "two_pass_bytes_per_step": step_bytes,
                      "achieved_gbs": achieved, "frac": achieved / hbm_peak},
        "roofline": {"bound": "hbm", "kernel": ("fine column kernel", "fine row kernel")[kid], "achieved": k_ach,
                     "peak": hbm_peak, "unit": "GB/s", "frac": k_ach / hbm_peak, "traffic": None,
                     "peak_kind": peak_kind, "avg_launch_us": 1e3 * prof_ms[kid] / max(1, prof_n[kid])},
        "clocks": clk, "gpu_launches": int(st.n_launches),
        "cpu_baseline": (None if args.no_cpu_baseline else
                         oracle_extrapolated(n, W["kz"], W["Rm"], T / N / S, S, N, 2)),
    }
    print(json.dumps(out), flush=True)
    kd.kd_destroy(ctx)


# ------------------------------------------------ batched sweep of independent instances
SWEEP_WL = {
    "workload": "rm_kz_sweep_parareal_32_slices",
    "slices": 32, "T": 8 * math.pi, "tol": 1e-6, "k_max": 32, "seed0": 1000,
    "recipe": "flow Roberts (even seed) / Galloway-Proctor (odd); Rm log-uniform [50, 3200]; n = 64 sqrt(Rm/50) "
              "rounded in log2 to [64, 512]; kz uniform [0.2, 1.5]; GP dt = 0.128/n, Roberts dt = 1.6/n; "
              "n_coarse = n/2; coarse dt = min(20 dt (GP) or 10 dt (Roberts), 2/n_coarse)",
}


def sweep_instances(kd, count, seed0):
    """The sweep's instances (parameters from kd_inputs.sweep_instance) and seeds."""
    import kd_inputs
    out = []
    for i in range(count):
        seed = seed0 + i
        q = kd_inputs.sweep_instance(seed)
        n, flow = q["n"], q["flow"]
        if flow == kd.KD_FLOW_GALLOWAY_PROCTOR:
            dt, ratio = 0.128 / n, 20
        else:
            dt, ratio = 1.6 / n, 10
        nc = n // 2
        dtc = min(ratio * dt, 2.0 / nc)     # explicit stability of the coarse grid
        out.append((seed, kd.make_instance(flow, n, q["kz"], q["Rm"], dt, nc, dtc), q))
    return out


def run_sweep(args):
    """The batched Rm / kz sweep: `--sweep-count` independent Parareal instances per rank in one
    kd_sweep_run call per step (ranks take disjoint seed ranges: weak scaling)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    import kd_inputs
    import paper_1902_00387_gb300 as kd
    kd.load()
    torch.cuda.init()
    W = dict(SWEEP_WL, count_per_rank=args.sweep_count)
    N, T = W["slices"], W["T"]
    insts = sweep_instances(kd, args.sweep_count, W["seed0"] + rank * args.sweep_count)
    b0_host = [torch.tensor(kd_inputs.initial_field(q.n, q.kz, seed)).pin_memory() for seed, q, _ in insts]
    b0_dev = [b.cuda() for b in b0_host]
    u_dev = [torch.zeros_like(b) for b in b0_dev]
    u_host = [torch.zeros_like(b).pin_memory() for b in b0_host]
    ins = [q for _, q, _ in insts]
    cache = os.path.join(tempfile.gettempdir(), "kd_tune_cache.json")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    # one prepared sweep for every step: groups, contexts and buffers made once, the fine
    # steps of recurring iterations replayed from captured CUDA graphs
    sw = kd.kd_sweep_create(ins, T, N)

    def solve(b0, out):
        s, res, st = kd.kd_sweep_exec(sw, b0, W["k_max"], W["tol"], u_final=out, tune_cache=cache)
        return s, res, st

    for _ in range(args.warmup):
        solve(b0_dev, u_dev)

    def timed(b0, out, steps, clocks=None):
        res = []
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        t = time.perf_counter()
        for i in range(steps):
            flush.fill_(float(i))
            torch.cuda.synchronize()
            res.append(solve(b0, out))
        torch.cuda.synchronize()
        el = time.perf_counter() - t
        ck = clocks.stop() if clocks else None
        if world > 1:
            tt = torch.tensor([el], dtype=torch.float64, device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            el = tt.item()
        return el, res, ck

    el, res, clk = timed(b0_dev, u_dev, args.steps, ClockSampler(local))
    s, results, st = res[-1]
    # serial-fine-equivalent work of one solve: every instance's N x S fine steps
    units = sum(3 * q.n ** 2 * N * r.n_fine_steps for q, r in zip(ins, results))
    value = units * world * args.steps / el / 1e6
    # fine work actually done and its two-pass algorithmic bytes
    fine_bytes = 0.0
    for q, r in zip(ins, results):
        cb, rb = col_row_bytes(q.n, 1)
        per_slice_step = 4 * (cb + rb)
        fine_bytes += sum(N - min(k - 1, N - 1) for k in range(1, r.k_con + 1)) * r.n_fine_steps * per_slice_step
    hbm_peak, peak_kind = peaks()
    achieved = fine_bytes / (st.ms_fine / 1e3) / 1e9
    e2e_value = None
    if not args.no_e2e:
        el_e2e, _, _ = timed(b0_host, u_host, max(1, args.steps // 2))
        e2e_value = units * world * max(1, args.steps // 2) / el_e2e / 1e6
    nbytes = sum(b.numel() * 16 for b in b0_host)
    ks = [r.k_con for r in results]
    by_n = {}
    for q, r in zip(ins, results):
        by_n.setdefault(q.n, []).append(r.k_con)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64 fine / f64 update", "data": "synthetic",
        "config": dict(W, l2="flushed between steps (512 MB write)",
                       parallelism="instances x slices in one batched launch per grid; ranks take disjoint seeds",
                       graphs="fine steps of each (iteration, active set) captured once, replayed in later steps"),
        "instances_by_n": {str(k): len(v) for k, v in sorted(by_n.items())},
        "k_con_by_n": {str(k): v for k, v in sorted(by_n.items())},
        "converged": sum(1 for r in results if r.status == kd.KD_OK), "k_con_max": max(ks),
        "phase_ms": {"fine": st.ms_fine, "coarse_and_update": st.ms_coarse, "total": st.ms_total},
        "fine_mdof_steps_per_s": st.fine_dof_steps / (st.ms_fine / 1e3) / 1e6,
        "roofline": {"bound": "hbm", "kernel": "fine phase (column + row kernels, increment gather/scatter)",
                     "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                     "traffic": None, "peak_kind": peak_kind},
        "clocks": clk,
        "e2e": ({"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}
                if e2e_value is not None else None),
        "gpu_launches": int(st.n_launches) * args.steps,
        "cpu_baseline": None,
    }
    kd.kd_sweep_destroy(sw)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# FP32 arithmetic rate from unit counts and clocks: 152 SMs x 128 FP32 lanes x 2 flops
# (fused multiply-add) x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12

def conv_roofline(n, S, batches, steps, stats):
    """ALU roofline of the convolution-form fine propagator: ~135 flops per kept mode and
    stage (the cross products with the 4 flow modes as 8 complex products and their sums,
    ~80; curl, ~18; stage update, ~36), i.e. 540 P^2 flops per slice-step, over the fine
    phase's device time."""
    P = 2 * (n // 3) + 1
    flops = 540.0 * P * P * S * sum(batches) * steps
    tf = flops / (sum(x.ms_fine for x in stats) / 1e3) / 1e12
    return {"bound": "alu", "kernel": "coarse_cluster_kernel<float, 4> as the fine convolution operator",
            "achieved": tf, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": tf / FP32_PEAK_TFLOPS,
            "traffic": None, "peak_kind": "derived from unit counts and the 2.07 GHz clock"}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ------------------------------------------------------------- shared set-up
class Env:
    """Rank, device, the library binding and the seeded input module of one bench process."""

    def __init__(self):
        import torch
        import torch.distributed as dist
        self.rank, self.world, self.local = dist_env()
        if self.world > 1:
            dist.init_process_group("nccl")
        torch.cuda.set_device(self.local)
        import __graft_entry__
        if self.rank == 0:
            __graft_entry__.build()
        if self.world > 1:
            dist.barrier()
        import kd_inputs
        import paper_1902_00387_gb300 as kd
        kd.load()
        torch.cuda.init()
        self.kd, self.I, self.torch, self.dist = kd, kd_inputs, torch, dist
        self.stream = torch.cuda.current_stream()

    def max_over_ranks(self, v):
        if self.world == 1:
            return v
        t = self.torch.tensor([v], dtype=self.torch.float64, device="cuda")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return t.item()

    def timed(self, fn, steps, clocks=None, flush=None):
        """Device time of `steps` calls of fn, each bracketed by CUDA events on the current
        stream; barrier and synchronize on both sides of the region."""
        torch = self.torch
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        res = []
        if self.world > 1:
            self.dist.barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        for i in range(steps):
            if flush is not None:
                flush.fill_(float(i))          # evict L2 between steps (buffer > 129 MB L2)
            ev[i][0].record(self.stream)
            res.append(fn())
            ev[i][1].record(self.stream)
        torch.cuda.synchronize()
        ck = clocks.stop() if clocks else None
        if self.world > 1:
            self.dist.barrier()
        return [x.elapsed_time(y) for x, y in ev], res, ck

    def close(self):
        if self.world > 1:
            self.dist.destroy_process_group()


# ------------------------------------------- Parareal, GP 128^2, 64 slices (the c2 solve)
def parareal_c2(args, env, embedded):
    """One Parareal solve of the 128^2 GP problem per step.  Returns the record of the
    line (`embedded`: the keys reported beside the default line, no e2e or CPU baseline)."""
    kd, torch = env.kd, env.torch
    stream = env.stream
    n, N, T = WL["n"], WL["slices"], WL["T"]
    fine_op = kd.KD_FINE_CONV if args.fine_operator == "conv" else kd.KD_FINE_FFT
    params = kd.make_params(kd.KD_FLOW_GALLOWAY_PROCTOR, n, WL["kz"], WL["Rm"], WL["dt_fine_max"], kd.KD_C64,
                            n_coarse=WL["n_coarse"], dt_coarse=WL["dt_coarse_max"], prec_coarse=kd.KD_C64,
                            fine_form=kd.KD_FINE_INCREMENT, fine_operator=fine_op)
    ctx = kd.kd_create(params, stream.cuda_stream)
    tune_ms = kd.kd_autotune(ctx, kd.KD_GRID_FINE, N, 3, os.path.join(tempfile.gettempdir(), "kd_tune_cache.json"))
    plan = kd.kd_get_plan(ctx, kd.KD_GRID_FINE)
    b0_host = torch.tensor(env.I.initial_field(n, WL["kz"], 1000 + env.rank)).pin_memory()
    b0_dev = b0_host.to("cuda")
    u_dev = torch.zeros((N + 1, 3, n, n), dtype=torch.complex128, device="cuda")
    u_host = torch.zeros((N + 1, 3, n, n), dtype=torch.complex128).pin_memory()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")

    def solve(b0, out):
        s, st = kd.kd_parareal_run(ctx, b0, T, N, WL["k_max"], WL["tol"], out)
        if s != kd.KD_OK:
            raise RuntimeError("Parareal did not converge: " + kd.kd_last_error(ctx))
        return st

    steps = args.steps if not embedded else max(3, min(args.steps, 5))
    for _ in range(args.warmup):
        solve(b0_dev, u_dev)
    # ---- timed region: device-resident inputs, no instrumentation
    launches0 = kd.kd_launch_count(ctx)
    ms, stats, clk = env.timed(lambda: solve(b0_dev, u_dev), steps, None if embedded else ClockSampler(env.local),
                               flush)
    launches = kd.kd_launch_count(ctx) - launches0
    # ---- kernel timing for the roofline: the same solve with every fine launch bracketed
    # by CUDA events on the context stream (separate from the timed region: the events
    # serialise the dependent launches)
    prof_steps = 2
    kd.kd_profile(ctx, 1)
    for _ in range(prof_steps):
        solve(b0_dev, u_dev)
    torch.cuda.synchronize()
    prof_ms, prof_n = kd.kd_profile_read(ctx)
    kd.kd_profile(ctx, 0)
    total_ms = env.max_over_ranks(sum(ms))
    ms_per_step = total_ms / steps
    units = units_per_solve()
    value = units * env.world * steps / (total_ms / 1e3) / 1e6
    st = stats[-1]

    e2e = None
    if not embedded:
        # end to end: host initial field in, all slice states back to host
        ms_e2e, _, _ = env.timed(lambda: solve(b0_host, u_host), max(2, steps // 2), flush=flush)
        e2e_total = env.max_over_ranks(sum(ms_e2e))
        d2h = (N + 1) * 3 * n * n * 16 + 8 * st.k_con + 8 * (N + 1) + 16
        e2e = {"value": units * env.world * len(ms_e2e) / (e2e_total / 1e3) / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": 3 * n * n * 16, "d2h_bytes_per_step": d2h}

    # ---- serial fine stepping of the same problem with the same kernels (complex64) and
    # with the complex128 kernels, the latter as the reference that separates the
    # Parareal error from FP32 round-off
    ser = torch.zeros_like(u_dev)
    kd.kd_fine_serial(ctx, b0_dev, T, N, ser)
    ms_ser, _, _ = env.timed(lambda: kd.kd_fine_serial(ctx, b0_dev, T, N, ser), 2)
    serial_ms = min(ms_ser)
    p128 = kd.make_params(kd.KD_FLOW_GALLOWAY_PROCTOR, n, WL["kz"], WL["Rm"], WL["dt_fine_max"], kd.KD_C128)
    ctx128 = kd.kd_create(p128, stream.cuda_stream)
    ser128 = torch.zeros_like(u_dev)
    kd.kd_fine_serial(ctx128, b0_dev, T, N, ser128)
    torch.cuda.synchronize()
    kd.kd_destroy(ctx128)
    rel = lambda a, b: (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item()
    solve(b0_dev, u_dev)
    torch.cuda.synchronize()
    err = rel(u_dev[-1], ser[-1])
    # error of every iterate against the complex64 and complex128 serial solutions (untimed)
    kd.kd_set_reference(ctx, ser[-1])
    st_ref = solve(b0_dev, u_dev)
    kd.kd_set_reference(ctx, ser128[-1])
    st_ref128 = solve(b0_dev, u_dev)
    kd.kd_set_reference(ctx, None)
    true_err = [float(st_ref.true_err[i]) for i in range(st_ref.k_con)]
    true_err128 = [float(st_ref128.true_err[i]) for i in range(st_ref128.k_con)]

    # ---- roofline of the dominant fine kernel, from the live event timing
    hbm_peak, peak_kind = peaks()
    S = st.n_fine_steps
    # fine-sweep batches over one solve: slices k-1..N-1 in iteration k
    batches = [N - min(k - 1, N - 1) for k in range(1, st.k_con + 1)]
    col_b = sum(col_row_bytes(n, b)[0] * 4 * S for b in batches) * prof_steps
    row_b = sum(col_row_bytes(n, b)[1] * 4 * S for b in batches) * prof_steps
    kid = 0 if prof_ms[0] >= prof_ms[1] else 1
    kbytes = (col_b, row_b)[kid]
    achieved = kbytes / (prof_ms[kid] / 1e3) / 1e9 if prof_ms[kid] > 0 else 0.0
    fine_units = 3 * n * n * S * sum(batches) * steps
    fine_rate = fine_units / (sum(x.ms_fine for x in stats) / 1e3) / 1e6
    if args.fine_operator == "fft":
        roof = {"bound": "latency (L2-resident)", "kernel": ("fine column kernel", "fine row kernel")[kid],
                "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": None, "algorithmic_bytes_per_launch": kbytes / max(1, prof_n[kid]), "peak_kind": peak_kind,
                "avg_launch_us": 1e3 * prof_ms[kid] / max(1, prof_n[kid]), "launches": prof_n[kid],
                "note": "the fine sweep's ~80 MB working set stays in the 129 MB L2; the HBM peak is the "
                        "reference the byte model is quoted against, not this kernel's bound"}
    else:
        roof = conv_roofline(n, S, batches, steps, stats)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": env.world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64 fine / f64 update", "data": "synthetic",
        "config": dict(WL, fine_steps_per_slice=S, coarse_steps_per_slice=st.n_coarse_steps,
                       l2="flushed between steps (512 MB write)", parallelism="time slices in one launch; "
                       "ranks solve independent instances", fine_plan=list(plan), fine_operator=args.fine_operator,
                       fine_plan_ms_per_step=tune_ms),
        "time_to_solution_ms": ms_per_step, "serial_fine_ms": serial_ms,
        "speedup_vs_serial_fine": serial_ms / ms_per_step, "k_con": st.k_con,
        "sigma": list(st.sigma[:st.k_con]), "err_vs_serial_fine": err, "true_err_by_iteration": true_err,
        "err_vs_serial_fine_c128": {
            "parareal_by_iteration": true_err128,
            "serial_fine_c64": rel(ser[-1], ser128[-1]),
            "note": "relative L2 error of the last slice state against the serial fine solution computed "
                    "with the complex128 kernels"},
        "growth_rate": st.growth_rate, "fine_mdof_steps_per_s": fine_rate,
        "phase_ms": {"fine": st.ms_fine, "coarse_and_update": st.ms_coarse},
        "roofline": roof,
        "gpu_launches": launches,
    }
    if not embedded:
        out["clocks"] = clk
        out["e2e"] = e2e
    kd.kd_destroy(ctx)
    return out


def run_parareal(args):
    env = Env()
    out = parareal_c2(args, env, embedded=False)
    if env.rank == 0 and not args.no_cpu_baseline:
        nsteps = 3 * out["config"]["fine_steps_per_slice"]
        v, el = oracle_sample(nsteps)
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": "%d RK443 fine steps (3 slices) of the 128^2 GP problem, serial, numpy "
                                         "FP64 oracle, %.1f s" % (nsteps, el)}
        try:
            out["cpu_baseline_all_cores"] = oracle_sample_all_cores(out["config"]["fine_steps_per_slice"])
        except Exception as e:   # the all-cores figure is context; its failure must not cost the line
            out["cpu_baseline_all_cores"] = {"error": "%s: %s" % (type(e).__name__, e)}
    if env.rank == 0:
        print(json.dumps(out), flush=True)
    env.close()


# ------------------------------------------------- the default line: the fine step, c5
# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the fine
# kernels, from one ncu capture of the warp-transform plan (6, 7) at 1024^2 x 16 slices
# (one fine step: the 4 stage launches of each kernel), averaged over the stages and
# scaled by 16 to a 256-slice launch (the traffic grows with the slices); keyed by the
# kernel's name as the bench reports it and its variant (column variant for the column
# kernel, row variant for the row kernel).  A variant without a capture of its current
# code reports null.
FINE_TRAFFIC = {
    ("fine row kernel", 7): 16 * (1196.97 + 1374.91 + 1021.99 + 785.88) / 4 * 1e6,
    ("fine column kernel", 6): 16 * (484.81 + 484.54 + 484.87 + 484.66) / 4 * 1e6,
}


E2E_CHUNK = 0    # chunks of the end-to-end host-buffer call: the library's graded plan (8 .. 48 fields)


def run_fine_step(args):
    env = Env()
    kd, torch = env.kd, env.torch
    W = FINE_WL
    n, B = W["n"], W["slices"]
    dt = fine_wl_dt()
    params = kd.make_params(kd.KD_FLOW_GALLOWAY_PROCTOR, n, W["kz"], W["Rm"], dt, kd.KD_C64)
    ctx = kd.kd_create(params, env.stream.cuda_stream)
    tune_ms = kd.kd_autotune(ctx, kd.KD_GRID_FINE, B, 2, os.path.join(tempfile.gettempdir(), "kd_tune_cache.json"))
    plan = kd.kd_get_plan(ctx, kd.KD_GRID_FINE)
    seeds = range(1000 + 8 * env.rank, 1008 + 8 * env.rank)
    base = torch.tensor(env.I.initial_batch(n, W["kz"], seeds), dtype=torch.complex64)
    x_dev = base.cuda().repeat(B // 8, 1, 1, 1)
    y_dev = torch.empty_like(x_dev)
    t0 = torch.arange(B, dtype=torch.float64, device="cuda") * (W["T"] / B)

    def step():
        kd.kd_fine_batched(ctx, x_dev, y_dev, t0, W["steps_per_call"], B)

    for _ in range(args.warmup):
        step()
    # ---- timed region: inputs resident in HBM (6.4 GB in, 6.4 GB out: larger than L2)
    launches0 = kd.kd_launch_count(ctx)
    ms, _, clk = env.timed(step, args.steps, ClockSampler(env.local))
    launches = kd.kd_launch_count(ctx) - launches0
    total_ms = env.max_over_ranks(sum(ms))
    ms_per_step = total_ms / args.steps
    units = 3 * n * n * B * W["steps_per_call"]
    value = units * env.world * args.steps / (total_ms / 1e3) / 1e6

    # ---- per-kernel timing for the roofline (a separate pass: the events serialise the
    # dependent launches)
    prof_calls = 2
    kd.kd_profile(ctx, 1)
    for _ in range(prof_calls):
        step()
    torch.cuda.synchronize()
    prof_ms, prof_n = kd.kd_profile_read(ctx)
    kd.kd_profile(ctx, 0)
    cb, rb = col_row_bytes(n, B)
    hbm_peak, peak_kind = peaks()
    kid = 0 if prof_ms[0] >= prof_ms[1] else 1
    kname = ("fine column kernel", "fine row kernel")[kid]
    avg_us = 1e3 * prof_ms[kid] / max(1, prof_n[kid])
    kbytes = (cb, rb)[kid]
    achieved = kbytes / (avg_us / 1e6) / 1e9
    stage_ms = (prof_ms[0] + prof_ms[1]) / prof_calls
    stage_bytes = 4 * (cb + rb) * W["steps_per_call"]
    traffic = FINE_TRAFFIC.get((kname, plan[kid]))

    # ---- a longer call: the same kernels over 8 steps (the conversions amortised)
    x2 = x_dev.clone()
    ms8, _, _ = env.timed(lambda: kd.kd_fine_batched(ctx, x2, x2, t0, 8, B), 2)
    del x2

    # ---- end to end: fields from pinned host memory in, results to pinned host memory out,
    # through the library's host-buffer call (chunks of E2E_CHUNK fields: the copy in of a
    # chunk, its step and the copy out of the previous chunk overlap)
    # The state of the method is the kept-mode square (|kx|, |ky| <= n/3, 683^2 of the 1024^2
    # coefficients): kd_fine_batched_host_kept moves only it across the host link (the line's
    # e2e); kd_fine_batched_host moves the whole [3][n][n] arrays (reported beside it).
    # The host link is shared with the machine's other GPUs: single calls now and then take
    # 2-4x as long while the copies alone slow down as much.  The value is the median call
    # (max over ranks); every call's time is listed beside it.
    t0_host = t0.cpu().numpy()
    e2e_reps = max(5, args.steps)

    def host_e2e(call, x_host):
        y_host = torch.empty_like(x_host).pin_memory()
        fn = lambda: call(ctx, x_host, y_host, t0_host, W["steps_per_call"], B, E2E_CHUNK)
        fn()
        ms_h, _, _ = env.timed(fn, e2e_reps)
        med = env.max_over_ranks(sorted(ms_h)[len(ms_h) // 2])
        del y_host
        return units * env.world / (med / 1e3) / 1e6, ms_h, x_host.numel() * x_host.element_size()

    idx = (torch.arange(-(n // 3), n // 3 + 1, device="cuda") % n)
    xk_host = x_dev[:, :, idx[:, None], idx[None, :]].contiguous().cpu().pin_memory()
    e2e_value, ms_e2e, nbytes = host_e2e(kd.kd_fine_batched_host_kept, xk_host)
    del xk_host
    xf_host = x_dev.cpu().pin_memory()
    full_value, ms_full, full_bytes = host_e2e(kd.kd_fine_batched_host, xf_host)
    del xf_host
    torch.cuda.synchronize()
    kd.kd_destroy(ctx)
    del x_dev, y_dev
    torch.cuda.empty_cache()

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": env.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": dict(W, dt_fine=dt, l2="inputs and outputs (6.4 GB each) larger than the 129 MB L2, no flush",
                       parallelism="all slices in one launch per kernel; ranks advance independent slice sets",
                       fine_plan=list(plan), fine_plan_ms_per_step=tune_ms),
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": kbytes, "avg_launch_us": avg_us, "launches": prof_n[kid],
                     "traffic_unit": "dram bytes per launch (ncu, 16-slice capture x 16)"},
        "fine_step_kernels": {
            "ms_per_step": stage_ms, "two_pass_bytes_per_step": stage_bytes,
            "achieved_gbs": stage_bytes / (stage_ms / 1e3) / 1e9,
            "frac": stage_bytes / (stage_ms / 1e3) / 1e9 / hbm_peak,
            "column_us_per_launch": 1e3 * prof_ms[0] / max(1, prof_n[0]),
            "row_us_per_launch": 1e3 * prof_ms[1] / max(1, prof_n[1]),
            "note": "the 4 column and 4 row stage launches of a step, event-timed (the prologue's inverse x "
                    "transform and the pack / unpack kernels of the call are outside these)"},
        "call_of_8_steps": {"ms": min(ms8), "mdof_steps_per_s": 8 * units / (min(ms8) / 1e3) / 1e6},
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                "call": "kd_fine_batched_host_kept: the fields' kept-mode squares [256][3][683][683] complex64 "
                        "from and to pinned host buffers, graded chunks (8, 16, 32, 48, 48, 48, 32, 16, 8 fields)",
                "ms_per_step": [round(v, 3) for v in ms_e2e], "stat": "median call"},
        "e2e_full_layout": {"value": full_value, "unit": UNIT, "h2d_bytes_per_step": full_bytes,
                            "d2h_bytes_per_step": full_bytes,
                            "call": "kd_fine_batched_host: whole [256][3][1024][1024] complex64 arrays, pinned host "
                                    "buffers, graded chunks (8, 16, 32, 48, 48, 48, 32, 16, 8 fields)",
                            "ms_per_step": [round(v, 3) for v in ms_full], "stat": "median call"},
        "gpu_launches": launches,
    }
    if env.rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = oracle_extrapolated(n, W["kz"], W["Rm"], dt, W["fine_steps_per_slice"], B, 2)
    if not args.no_parareal:
        c2 = parareal_c2(args, env, embedded=True)
        out["parareal_gp128"] = {k: c2[k] for k in (
            "time_to_solution_ms", "serial_fine_ms", "speedup_vs_serial_fine", "k_con", "sigma",
            "err_vs_serial_fine", "true_err_by_iteration", "err_vs_serial_fine_c128", "growth_rate",
            "fine_mdof_steps_per_s", "phase_ms", "roofline", "value", "unit", "steps")}
        out["parareal_gp128"]["config"] = c2["config"]
    if env.rank == 0:
        print(json.dumps(out), flush=True)
    env.close()


# ------------------------------------------------------------ small cases for ncu
def run_profile(args):
    """Small repeatable launches for profiling (ncu -k ... -s ... -c ...):
    --case fine: `--batch` seeded GP fields of side `--n` advanced by `--nsteps` fine steps,
        once to warm up and once more (the launches to capture), plan `--plan c,r`;
    --case parareal: one Parareal solve of the 128^2, 64-slice problem;
    --case coarse: the classical coarse propagator on one field (`--n-coarse`, `--nsteps`);
    --case gemm: the BF16 training GEMM `--gemm M,N,K` (`--engine` 0 tcgen05, 1 mma.sync).
    Prints the device time of the second call."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import kd_inputs
    import paper_1902_00387_gb300 as kd
    kd.load()
    torch.cuda.init()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    if args.case == "parareal":
        n, N, T = WL["n"], WL["slices"], WL["T"]
        p = kd.make_params(kd.KD_FLOW_GALLOWAY_PROCTOR, n, WL["kz"], WL["Rm"], WL["dt_fine_max"], kd.KD_C64,
                           n_coarse=WL["n_coarse"], dt_coarse=WL["dt_coarse_max"], prec_coarse=kd.KD_C64,
                           fine_form=kd.KD_FINE_INCREMENT)
        ctx = kd.kd_create(p)
        if args.plan:
            kd.kd_set_plan(ctx, kd.KD_GRID_FINE, *(int(v) for v in args.plan.split(",")))
        else:
            kd.kd_autotune(ctx, kd.KD_GRID_FINE, N, 2)
        b0 = torch.tensor(kd_inputs.initial_field(n, WL["kz"], 1000), device="cuda")
        e0, e1 = ev(), ev()
        e0.record()
        s, st = kd.kd_parareal_run(ctx, b0, T, N, WL["k_max"], WL["tol"])
        e1.record()
        torch.cuda.synchronize()
        print("parareal GP 128^2 x 64 slices: %.1f ms, k_con %d, plan %s" % (e0.elapsed_time(e1), st.k_con,
                                                                            kd.kd_get_plan(ctx)))
        kd.kd_destroy(ctx)
        return
    if args.case == "gemm":
        M, Nn, K = (int(v) for v in args.gemm.split(","))
        g = torch.Generator(device="cuda").manual_seed(1)
        A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
        Bt = torch.randn(Nn, K, device="cuda", generator=g).to(torch.bfloat16)
        C = torch.empty(M, Nn, device="cuda")
        kd.kd_gemm_bf16_tn(A, Bt, C, args.engine)
        e0, e1 = ev(), ev()
        e0.record()
        kd.kd_gemm_bf16_tn(A, Bt, C, args.engine)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        print("gemm %dx%dx%d engine %d: %.3f ms, %.1f TFLOP/s" % (M, Nn, K, args.engine, ms, 2.0 * M * Nn * K / ms / 1e9))
        return
    if args.case == "coarse":
        p = kd.make_params(kd.KD_FLOW_GALLOWAY_PROCTOR, args.n, args.kz, args.Rm, args.dt, kd.KD_C64,
                           n_coarse=args.n_coarse, dt_coarse=2.0 / args.n_coarse, prec_coarse=kd.KD_C64)
        ctx = kd.kd_create(p)
        if args.cluster:
            kd.kd_set_coarse_cluster(ctx, args.cluster)
        kd.kd_set_coarse_sync(ctx, args.sync)
        x = torch.tensor(kd_inputs.initial_batch(args.n, args.kz, [7]), dtype=torch.complex128, device="cuda")
        y = torch.empty_like(x)
        t0 = torch.zeros(1, dtype=torch.float64, device="cuda")
        kd.kd_coarse(ctx, x, y, t0, args.nsteps, 1)
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record()
        kd.kd_coarse(ctx, x, y, t0, args.nsteps, 1)
        e1.record()
        torch.cuda.synchronize()
        print("coarse N_C=%d steps=%d cluster=%d sync=%d: %.3f ms, %.3f us per stage" % (
            args.n_coarse, args.nsteps, args.cluster, args.sync, e0.elapsed_time(e1),
            e0.elapsed_time(e1) * 1000 / (4 * args.nsteps)))
        kd.kd_destroy(ctx)
        return
    p = kd.make_params(kd.KD_FLOW_GALLOWAY_PROCTOR, args.n, args.kz, args.Rm, args.dt, kd.KD_C64)
    ctx = kd.kd_create(p)
    if args.plan:
        c, r = (int(v) for v in args.plan.split(","))
        kd.kd_set_plan(ctx, kd.KD_GRID_FINE, c, r)
    # distinct seeds up to 64 fields; beyond, 8 seeded fields tiled
    nseed = args.batch if args.batch <= 64 else 8
    base = torch.tensor(kd_inputs.initial_batch(args.n, args.kz, range(nseed)), dtype=torch.complex64, device="cuda")
    x = base.repeat((args.batch + nseed - 1) // nseed, 1, 1, 1)[:args.batch].contiguous()
    t0 = torch.arange(args.batch, dtype=torch.float64, device="cuda") * 0.785
    kd.kd_fine_batched(ctx, x, x, t0, args.nsteps, args.batch)
    torch.cuda.synchronize()
    e0, e1 = ev(), ev()
    e0.record()
    kd.kd_fine_batched(ctx, x, x, t0, args.nsteps, args.batch)
    e1.record()
    torch.cuda.synchronize()
    print("n=%d batch=%d steps=%d plan %s: %.3f ms" % (args.n, args.batch, args.nsteps, kd.kd_get_plan(ctx),
                                                       e0.elapsed_time(e1)))
    kd.kd_destroy(ctx)


# --------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-parareal", action="store_true",
                    help="default line: leave out the GP 128^2 Parareal solve reported beside it")
    ap.add_argument("--no-e2e", action="store_true", help="--config sweep: skip the end-to-end (host buffer) solves")
    ap.add_argument("--config", default="fine-step",
                    choices=["fine-step", "parareal", "learned", "sweep", "large", "steppers", "coarse-sweep",
                             "coarse-sweep-roberts", "profile"],
                    help="fine-step: one fine step of the 256 slices of the GP 1024^2 problem (default); "
                         "parareal: Parareal on the GP 128^2 problem; learned: learned vs classical coarse, GP 256^2; "
                         "sweep: batched independent instances (Rm / kz sweep); large: Parareal on GP 1024^2, "
                         "256 slices; steppers: RK111 / RK222 / RK443 accuracy per work; coarse-sweep: N_C study on "
                         "the GP 128^2 problem; coarse-sweep-roberts: N_C study at Rm 512, N_F 160; profile: small "
                         "cases for ncu (--case)")
    ap.add_argument("--sweep-count", type=int, default=32, help="instances per rank of --config sweep")
    ap.add_argument("--fine-operator", default="fft", choices=["fft", "conv"],
                    help="fft: the pseudo-spectral fine step (the workload's definition); conv: the same operator "
                         "as the exact spectral convolution in one persistent launch")
    # --config profile
    ap.add_argument("--case", default="fine", choices=["fine", "parareal", "coarse", "gemm"])
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--nsteps", type=int, default=1)
    ap.add_argument("--kz", type=float, default=0.57)
    ap.add_argument("--Rm", type=float, default=1e4)
    ap.add_argument("--dt", type=float, default=1e-3)
    ap.add_argument("--plan", default=None, help="column,row variant of the fine kernels")
    ap.add_argument("--n-coarse", type=int, default=128)
    ap.add_argument("--cluster", type=int, default=0, help="blocks per cluster of the coarse solver (0: default)")
    ap.add_argument("--sync", type=int, default=0, help="coarse halo exchange: 0 cluster barrier, 1 point-to-point")
    ap.add_argument("--gemm", default="4096,4096,4096", help="M,N,K of a BF16 GEMM to run")
    ap.add_argument("--engine", type=int, default=0, help="GEMM engine: 0 tcgen05, 1 mma.sync")
    args = ap.parse_args()
    if args.config == "profile":
        run_profile(args)
        return
    # the measured lines take at least 3 warm-up steps; the sweep study, whose 256-instance
    # solves take minutes, may take fewer (it reports the number it used)
    if args.config != "sweep":
        args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return
    runs = {"fine-step": run_fine_step, "parareal": run_parareal, "learned": run_learned, "sweep": run_sweep,
            "large": run_large, "steppers": run_steppers, "coarse-sweep": run_coarse_sweep,
            "coarse-sweep-roberts": run_roberts_coarse_sweep}
    runs[args.config](args)


if __name__ == "__main__":
    main()
