#!/usr/bin/env python3
"""Benchmark: Kob-Andersen binary LJ, N = 32 000, rho = 1.2, one GB300.

Workload (the 32k configuration): lattice + 0.05 jitter start at T = 2.0,
2000 Nose-Hoover steps to T = 0.8 (set-up, untimed), then NVE at dt = 0.005
with a cell + Verlet list whose force-list skin is 0.3 (rebuilt on the
device when any particle has moved more than skin/2; the autotuner may add an
outer list that the force list is pruned from). Other lines: --workload ka1k
(N = 1000 on the all-FP64 path, NVE from the lattice start at T = 2.0),
ka1m (10^6 particles, Nose-Hoover at T = 0.5, with the cost of the g(r) and
MSD calls reported separately), ka8m (8*10^6, quench 2.0 -> 0.45 then NVE,
with the device footprint), ensemble (512 replicas in one launch; with N
ranks the replicas are split over them by a greedy N-balanced partition),
ladder (the paper's cooling run sequence, 8 replicas of N = 1000 in one
launch).

One bench step = one persistent launch that advances the system 100 MD steps
(force + velocity Verlet + reductions + every list rebuild the dynamics
triggers), i.e. one md_step_nve(dt, 100) call. --steps K timed steps follow
--warmup W untimed ones; the default K = 100 covers the configuration's
10 000 NVE steps. L2 is flushed (a 256 MB write) between timed steps.

value     = atom-steps/s of the mixed-precision path (ka1k: FP64),
            device-timed (CUDA events on the system's stream), inputs
            resident in HBM; with N ranks, all ranks' atoms over the slowest
            rank's time.
e2e       = the same metric through the public C ABI with host buffers:
            md_set_state(host) + md_step_nve(100, thermo log to host) +
            md_get_state(host) per step.
drift     = slope of E_tot/N against t over the timed NVE window, with a
            moving-block bootstrap error; fp64 = the all-FP64 GPU path on the
            same protocol and the same window, with its drift;
            drift_equal_or_better = the metric's condition (mixed drift not
            larger than the FP64 drift beyond two combined error bars).
roofline  = FP32 issue bound ("alu") of the persistent kernel: algorithmic
            FLOPs per launch / launch time against 2*128*SMs*f_max.
cpu_baseline = the FP64 oracle (plain C, all pairs) on a bounded sample (a
            few MD steps of the same system) on every host core, with the
            one-thread rate beside it.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "atom-steps/s and pair-evals/s (mixed vs FP64 GPU) at equal NVE energy drift"
UNIT = "atom-steps/s"
N = 32000
SEED = 2
T_START, T_NVT = 2.0, 0.8
NVT_STEPS = 2000
CHUNK = 100
LOG_EVERY = 10
# counting convention for the pair loop (per list entry)
FLOP_PAIR_IN = 26   # interacting entry: dr 3, r^2 5, rcp 1, r^-6 2, sigma^6 r^-6 1, force 4, accumulate 6, energy 4
FLOP_PAIR_OUT = 8   # rejected entry: dr 3, r^2 5 (fixed-point minimum image is integer arithmetic)
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0


def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="kamd_clocks_", suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait(timeout=5)
        with open(self.path) as f:
            rec = parse_clock_samples(f)
        os.unlink(self.path)
        return rec


def parse_clock_samples(lines):
    """Median SM clock, maximum clock and every throttle reason seen, from nvidia-smi CSV rows
    (index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap)."""
    rows = []
    for line in lines:
        f = [x.strip() for x in line.split(",")]
        if len(f) >= 9 and f[1].replace(".", "").isdigit():
            rows.append(f)
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    sm = np.array([float(r[1]) for r in rows])
    smax = max(float(r[2]) for r in rows)
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": reasons, "samples": len(rows)}


def max_over_ranks(x, dist, device="cpu"):
    """Largest value of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, dist, device="cuda"):
    """Sum of x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(world, n_per_rank, md_steps, max_seconds):
    """Atom-steps/s of the whole job: every rank advances its own replica."""
    return world * n_per_rank * md_steps / max_seconds


def drift_per_tau(log, dt):
    """Least-squares slope of E_tot/N against time (energy per particle per tau) and the RMS
    fluctuation about it."""
    d = drift_stats(log, dt)
    return d["slope"], d["rms"]


def drift_stats(log, dt):
    """Drift of E_tot/N (first replica) over the logged window: slope, moving-block bootstrap error
    of the slope, RMS fluctuation about the fit, window length in steps."""
    from paper_2001_07089_gb300 import analysis
    e = np.asarray(log["etot_per_n"][:, 0], dtype=np.float64)
    st = np.asarray(log["step"][:, 0], dtype=np.float64)
    if len(e) < 4:
        return {"slope": None, "err": None, "rms": None, "window_steps": 0}
    d = analysis.drift_fit(st * dt, e)
    return {"slope": d["slope"], "err": d["err"], "rms": d["rms"], "window_steps": int(st[-1] - st[0])}


def drift_equal_or_better(mixed, fp64, k=2.0):
    """The metric's condition: the mixed path's drift magnitude is not larger than the FP64 path's
    beyond k combined error bars. None when either drift is missing."""
    if not mixed or not fp64 or mixed.get("slope") is None or fp64.get("slope") is None:
        return None
    sig = float(np.hypot(mixed["err"], fp64["err"]))
    return bool(abs(mixed["slope"]) <= abs(fp64["slope"]) + k * sig)


def partition_replicas(n_per, world):
    """Greedy N-balanced split of independent replicas over `world` ranks: largest replica first,
    each to the rank with the least load so far (lowest rank on ties). Returns one sorted index
    list per rank."""
    n_per = [int(x) for x in n_per]
    order = sorted(range(len(n_per)), key=lambda r: (-n_per[r], r))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for r in order:
        k = min(range(world), key=lambda q: (load[q], q))
        parts[k].append(r)
        load[k] += n_per[r]
    return [sorted(p) for p in parts]


WORKLOADS = {
    "ka1k": dict(kind="single", n=1000, seed=1, T0=2.0, T=None, setup_nvt=0, timed="nve", skin=0.3, prec="fp64",
                 desc="ka1k: Kob-Andersen 80:20, N=1000, rho=1.2, L=9.4104, 10^3 lattice+0.05 jitter, Maxwell-"
                      "Boltzmann T=2.0, NVE dt=0.005 on the all-FP64 path (no bath stage); force-list skin 0.3; "
                      "one bench step = 100 MD steps (--steps 10 = the configuration's 1000 steps)"),
    "ka32k": dict(kind="single", n=32000, seed=2, T0=2.0, T=0.8, setup_nvt=2000, timed="nve", skin=0.3,
                  desc="ka32k: Kob-Andersen 80:20, N=32000, rho=1.2, L=29.876, lattice+0.05 jitter at T=2.0, "
                       "2000 Nose-Hoover steps to T=0.8 (untimed), then NVE dt=0.005; cell + Verlet list, force-list skin 0.3 (any outer list autotuned) "
                       "rebuilt on device; one bench step = 100 MD steps"),
    "ka1m": dict(kind="single", n=1_000_000, seed=3, T0=0.5, T=0.5, setup_nvt=200, timed="nvt",
                 desc="ka1m: Kob-Andersen 80:20, N=10^6, rho=1.2, L=94.104, 100^3 lattice+0.05 jitter at T=0.5, "
                      "Nose-Hoover NVT at T=0.5 dt=0.005 (200 untimed steps, then timed); one bench step = 100 MD steps"),
    "ka8m": dict(kind="single", n=8_000_000, seed=5, T0=2.0, T=0.45, setup_nvt=200, pre_nvt=(2.0, 200),
                 timed="nve",
                 desc="ka8m: Kob-Andersen 80:20, N=8*10^6, rho=1.2, L=188.207, 200^3 lattice+0.05 jitter at T=2.0, "
                      "200 Nose-Hoover steps at T=2.0 then an instant quench (200 steps at T=0.45), untimed; then NVE "
                      "dt=0.005; one bench step = 100 MD steps"),
    "ensemble": dict(kind="ensemble", nrep=512, seed=4, T0=2.0, setup_nvt=200, timed="nvt",
                     desc="ensemble: 512 independent KA replicas in one persistent launch, N per replica uniform "
                          "over {250,500,1000,2000,4000,8000}, rho=1.2, per-replica Nose-Hoover at T uniform in "
                          "[0.45,2.0], dt=0.005; one bench step = 100 MD steps of every replica"),
    "ladder": dict(kind="ladder", nrep=8, n=1000, seed=6, T0=5.0, timed="ladder",
                   temps=[5.0, 4.0, 3.0, 2.0, 1.0, 0.8, 0.6, 0.55, 0.5, 0.475, 0.466],
                   desc="ladder: the cooling run sequence on 8 independent KA replicas of N=1000 (rho=1.2, L=9.4104) "
                        "in one launch: lattice+0.05 jitter, 200 steps of the stochastic bath at T=5.0 (untimed), "
                        "then per temperature T=5.0, 4.0, 3.0, 2.0, 1.0, 0.8, 0.6, 0.55, 0.5, 0.475, 0.466 one "
                        "bench step of the stochastic bath (redraw every 50 steps), one of NVE and one NVE "
                        "production step, dt=0.005; one bench step = 100 MD steps of every replica; e2e = NVE "
                        "launches of the same batch"),
}


def setup_system(kamd, wl, prec, device, wk=None, subset=None):
    """Build, start and equilibrate the workload's system; returns (system, n_total, T_target).
    subset: replica indices of the ensemble this rank runs (all when None)."""
    wk = wk or WORKLOADS["ka32k"]
    if wk["kind"] == "single":
        n = wk["n"]
        L = wl.box_length(n)
        types = wl.ka_types(n, wk["seed"])
        s = kamd.System(n, L, types, wl.KA_EPS, wl.KA_SIG, wl.KA_RC, wl.KA_MASS, wl.SKIN, prec)
        T = np.array([wk["T"]])
    elif wk["kind"] == "ladder":
        n_per = [wk["n"]] * wk["nrep"]
        L = wl.box_length(wk["n"])
        types = np.concatenate([wl.ka_types(wk["n"], wk["seed"] * 100003 + r) for r in range(wk["nrep"])])
        s = kamd.System(n_per, [L] * wk["nrep"], types, wl.KA_EPS, wl.KA_SIG, wl.KA_RC, wl.KA_MASS, wl.SKIN, prec)
        n = wk["n"] * wk["nrep"]
        T = np.full(wk["nrep"], wk["T0"])
    else:
        spec = wl.ensemble(wk["nrep"], wk["seed"])
        idx = list(range(len(spec.n))) if subset is None else list(subset)
        s = kamd.System(spec.n[idx], spec.L[idx], np.concatenate([spec.types[r] for r in idx]), wl.KA_EPS, wl.KA_SIG,
                        wl.KA_RC, wl.KA_MASS, wl.SKIN, prec)
        n = int(spec.n[idx].sum())
        T = spec.T[idx]
    s.init_lattice(wk["T0"], 0.05, wk["seed"])
    if "pre_nvt" in wk:  # a first bath stage before the quench to T
        T0, k0 = wk["pre_nvt"]
        s.step_nvt(wl.DT, k0, np.full_like(T, T0), kind=kamd.MD_NVT_NOSE_HOOVER, param=100 * wl.DT)
    if wk["kind"] == "ladder":  # equilibrate at the top of the ladder with the stochastic bath
        s.step_nvt(wl.DT, 200, T, kind=kamd.MD_NVT_RESAMPLE, param=50, seed=wk["seed"])
    elif wk["setup_nvt"] > 0:
        s.step_nvt(wl.DT, wk["setup_nvt"], T, kind=kamd.MD_NVT_NOSE_HOOVER, param=100 * wl.DT)
    return s, n, T


def analysis_cost(torch, s, reps=3):
    """Wall time of the analysis calls of the 10^6 configuration (partial g(r): 400 bins of 0.01 up to
    4 sigma; per-type MSD), each a synchronous call through the C ABI, best of `reps`."""
    out = {}
    for name, fn in (("rdf_ms", lambda: s.rdf(0.01, 400, reset=True)), ("msd_ms", lambda: s.msd())):
        best = None
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            dt_ = (time.perf_counter() - t0) * 1e3
            best = dt_ if best is None else min(best, dt_)
        out[name] = best
    return out


def timed_chunks(torch, s, dt, steps, warmup, flush, log_every=LOG_EVERY, step=None):
    """Time `steps` calls of `step(CHUNK, log_every)` (default: NVE) with CUDA events, L2 flushed between.
    Returns (seconds per call, the thermo log, the library's kernel launches during the timed calls)."""
    step = step or (lambda k, le: s.step_nve(dt, k, log_every=le))
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        step(CHUNK, 0)
    torch.cuda.synchronize()
    k0 = s.info()["kernel_launches"]  # outside the timed region
    logs, times = [], []
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        ev0[k].record(stream)
        logs.append(step(CHUNK, log_every))
        ev1[k].record(stream)
    torch.cuda.synchronize()
    times = [ev0[k].elapsed_time(ev1[k]) * 1e-3 for k in range(steps)]
    log = np.concatenate(logs, axis=0)
    return np.array(times), log, s.info()["kernel_launches"] - k0


def run_e2e(torch, kamd, s, dt, steps, T=None):
    """Public API with host buffers: set_state(host) + step (log to host) + get_state(host). The host
    buffers are pinned (page-locked) memory, as a caller streaming states would allocate them."""
    pos0, vel0, _ = s.get_state()
    n3 = (s.n_total, 3)

    def pinned(shape, dtype, init=None):
        t = torch.empty(int(np.prod(shape)) * np.dtype(dtype).itemsize, dtype=torch.uint8, pin_memory=True)
        a = t.numpy().view(dtype).reshape(shape)
        a[...] = 0 if init is None else init
        return a, t  # keep the tensor alive with the view

    (pos, tp), (vel, tv) = pinned(n3, np.float64, pos0), pinned(n3, np.float64, vel0)
    img, ti = pinned(n3, np.int32)
    nlog = CHUNK // LOG_EVERY
    log, tl = pinned((nlog * s.nrep,), kamd.THERMO_DTYPE)
    h = s.handle
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        kamd.md_set_state(h, pos, vel)
        if T is None:
            kamd.md_step_nve(h, dt, CHUNK, log, LOG_EVERY)
        else:
            kamd.md_step_nvt(h, dt, CHUNK, T, kamd.MD_NVT_NOSE_HOOVER, 100 * dt, 0, log, LOG_EVERY)
        kamd.md_get_state(h, pos, vel, img, 0)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    h2d = 2 * 3 * 8 * s.n_total
    d2h = (2 * 3 * 8 + 3 * 4) * s.n_total + log.nbytes
    return el, h2d, d2h


def kernel_sources_digest():
    """sha256 over the CUDA sources of the library (sorted by name)."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2001_07089_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()


def profiled_traffic(workload, tuning):
    """DRAM bytes (read + write) per launch of the persistent kernel, from the committed ncu summary
    of this workload, when it was taken on the current kernel sources with the same tuning; else None."""
    path = os.path.join(ROOT, "profiles", f"md_persistent_{workload}.md")
    if not os.path.exists(path):
        return None
    fields = {}
    with open(path) as f:
        for line in f:
            if line.startswith("- `") and "`: " in line:
                k, v = line[3:].split("`: ", 1)
                fields[k] = v.strip().strip("`")
    try:
        t = fields.get("tuning", "").split(",")
        want = [tuning["threads_per_atom"], tuning["block_size"], tuning["skin"], tuning["skin_outer"]]
        same = (fields.get("kernel_sources_sha256") == kernel_sources_digest() and len(t) == 4
                and all(abs(float(a) - float(b)) < 1e-9 for a, b in zip(t, want)))
        return float(fields["dram_bytes_per_launch"]) if same else None
    except (KeyError, ValueError):
        return None


def host_threads():
    """Host cores the oracle may use (its threaded force sum), at most 64."""
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    return max(1, min(64, n))


def cpu_baseline(wl, seconds_target=12.0):
    """The oracle as it stands (all-pairs FP64) on a few MD steps of the same N = 32 000 system: on
    one thread (the plain oracle) and on every host core (its threaded force sum)."""
    import oracle
    L = wl.box_length(N)
    types = wl.ka_types(N, SEED).astype(np.int32)
    params = oracle.Params(wl.KA_EPS, wl.KA_SIG, wl.KA_RC, wl.KA_MASS)
    pos, vel = oracle.init_lattice(N, L, T_START, SEED)
    t0 = time.perf_counter()
    f, _, _ = oracle.forces(pos, types, params, L)
    t_force = time.perf_counter() - t0
    n1 = max(1, min(10, int(0.5 * seconds_target / max(t_force, 1e-3)) - 1))
    t0 = time.perf_counter()
    oracle.run(pos, vel, types, params, L, wl.DT, n1, forces_in=f, log_every=0)
    v1 = N * n1 / (time.perf_counter() - t0)
    cores = host_threads()
    nall = max(1, min(100, int(0.5 * seconds_target * v1 * cores * 0.7 / N)))
    oracle.set_threads(cores)
    try:
        t0 = time.perf_counter()
        oracle.run(pos, vel, types, params, L, wl.DT, nall, forces_in=f, log_every=0)
        vall = N * nall / (time.perf_counter() - t0)
    finally:
        oracle.set_threads(1)
    return {"value": vall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{nall} velocity-Verlet steps of the N=32000 system, all-pairs FP64 C oracle on {cores} "
                      f"threads (per-thread force arrays added in thread order); on 1 thread: {n1} steps",
            "value_1_thread": v1}


def reference_arm(args, rank, world):
    """The tier's reference arm: the oracle as it stands (all-pairs FP64 C, its threaded force sum on
    every host core), one bench step = one MD step of the N = 32 000 system. Rank 0 only."""
    import torch.distributed as dist  # noqa: F401
    from paper_2001_07089_gb300 import workloads as wl
    if rank != 0:
        return
    import oracle
    L = wl.box_length(N)
    types = wl.ka_types(N, SEED).astype(np.int32)
    params = oracle.Params(wl.KA_EPS, wl.KA_SIG, wl.KA_RC, wl.KA_MASS)
    pos, vel = oracle.init_lattice(N, L, T_START, SEED)
    cores = host_threads()
    oracle.set_threads(cores)
    try:
        f, _, _ = oracle.forces_threads(pos, types, params, L, cores)
        st = {"pos": pos, "vel": vel, "forces": f}
        for _ in range(args.warmup):
            st = oracle.run(st["pos"], st["vel"], types, params, L, wl.DT, 1, forces_in=st["forces"], log_every=0)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            st = oracle.run(st["pos"], st["vel"], types, params, L, wl.DT, 1, forces_in=st["forces"], log_every=0)
        el = time.perf_counter() - t0
    finally:
        oracle.set_threads(1)
    v = N * args.steps / el
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic",
                      "config": {"workload": "ka32k: KA 80:20 N=32000 rho=1.2, NVE dt=0.005; one bench step = one "
                                             "oracle MD step (all pairs)"},
                      "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                       "sample": f"{args.steps} all-pairs velocity-Verlet steps of N=32000 on "
                                                 f"{cores} threads"},
                      "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kamd", choices=["kamd", "reference"])
    ap.add_argument("--workload", default="ka32k", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tuning", default=None,
                    help="fixed tuning 'threads_per_atom,block_size,skin,skin_outer' instead of the autotuner")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="timed bench steps of the all-FP64 arm (default: --steps for ka32k, 0 otherwise)")
    args = ap.parse_args()
    rank, world, local = env_rank()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    wk = WORKLOADS[args.workload]

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2001_07089_gb300 import kamd
    from paper_2001_07089_gb300 import workloads as wl
    kamd.load()
    dev = torch.cuda.current_device()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def stepper(sys_, T):
        if wk["timed"] == "nve":
            return lambda k, le: sys_.step_nve(wl.DT, k, log_every=le)
        if wk["timed"] == "ladder":
            # bench step j: stage j % 3 (bath, NVE, production) at temperature j // 3 of the ladder
            state = {"j": 0}

            def ladder_step(k, le):
                j = state["j"]
                state["j"] += 1
                Tk = wk["temps"][(j // 3) % len(wk["temps"])]
                if j % 3 == 0:
                    return sys_.step_nvt(wl.DT, k, Tk, kind=kamd.MD_NVT_RESAMPLE, param=50, seed=wk["seed"] + j,
                                         log_every=le)
                return sys_.step_nve(wl.DT, k, log_every=le)
            return ladder_step
        return lambda k, le: sys_.step_nvt(wl.DT, k, T, kind=kamd.MD_NVT_NOSE_HOOVER, param=100 * wl.DT,
                                           log_every=le)

    # ---- the measured path (mixed precision; ka1k: the configuration's FP64). Every rank runs its own
    # system; the ensemble's replicas are split over the ranks (greedy N-balanced partition).
    prec = wk.get("prec", "mixed")
    subset = None
    if wk["kind"] == "ensemble":
        spec_all = wl.ensemble(wk["nrep"], wk["seed"])
        subset = partition_replicas(spec_all.n, world)[rank]
    s, n_sys, T = setup_system(kamd, wl, prec, dev, wk, subset=subset)
    if args.tuning:
        t4 = args.tuning.split(",")
        s.set_tuning(threads_per_atom=int(t4[0]), block_size=int(t4[1]), skin=float(t4[2]), skin_outer=float(t4[3]))
    elif not args.no_autotune:
        # the configuration's force-list skin (ka32k: 0.3) is kept; the rest is searched
        s.autotune(wl.DT, probe_steps=200 if n_sys < 200000 else 60, skin=wk.get("skin"))
    tuning = s.tuning
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    rebuilds0 = s.info()["rebuilds"]
    clocks = Clocks(dev)
    clocks.start()
    times, log, launches = timed_chunks(torch, s, wl.DT, args.steps, args.warmup, flush, step=stepper(s, T))
    clk = clocks.stop()
    total = max_over_ranks(float(times.sum()), dist, "cuda")
    n_job = int(round(sum_over_ranks(n_sys, dist))) if dist else n_sys
    info = s.info()
    pairs = s.count_pairs()
    entries = info["list_entries"]
    pairs_job = sum_over_ranks(pairs, dist) if dist else pairs
    drift_main = drift_stats(log, wl.DT) if wk["timed"] == "nve" else None
    value = n_job * CHUNK * args.steps / total
    pair_evals = (sum_over_ranks(entries, dist) if dist else entries) * CHUNK * args.steps / total
    flop_step = FLOP_PAIR_IN * 2 * pairs + FLOP_PAIR_OUT * (entries - 2 * pairs)
    launch_s = float(times.sum()) / args.steps
    achieved = flop_step * CHUNK / launch_s / 1e12
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak = 2 * FP32_LANES_PER_SM * nsm * SM_MAX_MHZ * 1e6 / 1e12
    # the force phase alone (md_time_forces), on the final state: the FP32 roofline of the force kernel
    t_force = s.time_forces(100 if n_sys < 200000 else 20)
    force_phase = {"seconds_per_eval": t_force, "achieved": flop_step / t_force / 1e12, "peak": peak,
                   "unit": "TFLOP/s", "frac": flop_step / t_force / 1e12 / peak,
                   "entries": entries, "pairs_within_cutoff": pairs,
                   "note": "md_time_forces: pair sums over the force list and force stores of a step, no energies "
                           "and no velocity/position update, each evaluation closed by a grid barrier; "
                           "FLOPs = 26 per entry within r_c + 8 per other entry"}
    # the list build alone (md_time_lists), at the same state; its share of the timed steps follows
    # from the rebuilds those steps made (warm-up steps included, which the timed steps dominate)
    builds = info["rebuilds"] - rebuilds0
    t_list = s.time_lists(10 if n_sys < 200000 else 4)
    md_steps = CHUNK * (args.steps + args.warmup)
    single = wk["kind"] == "single"  # replicas of a batch rebuild separately: no single count
    list_build = {"seconds_per_build": t_list, "builds_per_md_step": builds / md_steps if single else None,
                  "share_of_step": t_list * builds / md_steps / (launch_s / CHUNK) if single else None,
                  "note": "md_time_lists: the Verlet-list build of a rebuild (after the cell sort) repeated "
                          "inside one launch; share = seconds per build x builds per MD step / seconds per MD "
                          "step of the timed launches"}
    analysis = analysis_cost(torch, s) if args.workload == "ka1m" else None
    device_bytes = info["device_bytes"]
    e2e = None
    if not args.no_e2e:
        e2e_steps = max(3, min(args.steps, 20))
        e2e_el, h2d, d2h = run_e2e(torch, kamd, s, wl.DT, e2e_steps, None if wk["timed"] in ("nve", "ladder") else T)
        e2e_el = max_over_ranks(e2e_el, dist, "cuda")
        e2e = {"value": n_job * CHUNK * e2e_steps / e2e_el, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}
    s.close()

    # ---- all-FP64 GPU path on the same protocol and window (the context of the metric: mixed vs FP64
    # at equal or better drift)
    fp64 = None
    k64 = args.fp64_steps if args.fp64_steps is not None else (args.steps if args.workload == "ka32k" else 0)
    if rank == 0 and k64 > 0 and prec == "mixed":
        s64, _, T64 = setup_system(kamd, wl, "fp64", dev, wk, subset=subset)
        if not args.no_autotune:
            s64.autotune(wl.DT, probe_steps=50 if n_sys < 200000 else 10, skin=wk.get("skin"))
        t64, log64, _ = timed_chunks(torch, s64, wl.DT, k64, 1, flush, step=stepper(s64, T64))
        d64 = drift_stats(log64, wl.DT) if wk["timed"] == "nve" else None
        fp64 = {"value": n_sys * CHUNK * k64 / float(t64.sum()), "unit": UNIT, "timed_md_steps": CHUNK * k64,
                "drift_per_particle_per_tau": d64["slope"] if d64 else None,
                "drift_err": d64["err"] if d64 else None,
                "drift_window_steps": d64["window_steps"] if d64 else None,
                "etot_fluct_per_particle": d64["rms"] if d64 else None,
                "tuning": s64.tuning}
        s64.close()

    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    cpu = None if args.no_cpu_baseline else cpu_baseline(wl)
    eq_better = drift_equal_or_better(drift_main, {"slope": fp64["drift_per_particle_per_tau"],
                                                   "err": fp64["drift_err"]} if fp64 else None)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "strong" if wk["kind"] == "ensemble" else "weak",
        "vs_baseline": None, "dtype": "f64" if prec == "fp64" else "f32", "data": "synthetic",
        "config": {"workload": wk["desc"], "n": n_job, "md_steps_per_bench_step": CHUNK,
                   "timed_md_steps": CHUNK * args.steps,
                   "precision": ("FP64 positions, velocities, forces and pair math" if prec == "fp64" else
                                 "mixed: 64-bit fixed-point positions, FP32 velocities/forces/pair math, "
                                 "FP64 reductions"),
                   "l2": "flushed between timed steps (256 MB write)", "tuning": tuning,
                   "parallelism": ("replicas split over ranks (greedy N-balanced)" if wk["kind"] == "ensemble"
                                   else "replicas only") if world > 1 else "single GPU"},
        "pair_evals_per_s": pair_evals,
        "useful_pair_evals_per_s": 2 * pairs_job * CHUNK * args.steps / total,
        "list_entries": entries, "pairs_within_cutoff": pairs,
        "drift_per_particle_per_tau": drift_main["slope"] if drift_main else None,
        "drift_err": drift_main["err"] if drift_main else None,
        "drift_window_steps": drift_main["window_steps"] if drift_main else None,
        "etot_fluct_per_particle": drift_main["rms"] if drift_main else None,
        "drift_note": ("slope of E_tot/N against t over the timed NVE window (thermo every 10 steps); err = "
                       "moving-block bootstrap of the residuals (one run: does not include run-to-run scatter)"),
        "fp64": fp64,
        "mixed_over_fp64": (value / world) / fp64["value"] if fp64 else None,
        "drift_equal_or_better": eq_better,
        "drift_equal_or_better_rule": "|d_mixed| <= |d_fp64| + 2 * hypot(err_mixed, err_fp64)",
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": profiled_traffic(args.workload, tuning),
                     "frac_at_measured_clock": (achieved / (peak * clk["sm_mhz"] / SM_MAX_MHZ)
                                                if clk.get("sm_mhz") else None),
                     "kernel": f"md_persistent<{'fp64' if prec == 'fp64' else 'mixed'}> (one launch = 100 MD steps)",
                     "peak_note": "FP32 FMA: 2 flops x 128 lanes x SMs x 2070 MHz (recipe unit counts and max clock)"},
        "force_phase": force_phase,
        "list_build": list_build,
        "analysis_ms": analysis,
        "device_bytes": device_bytes,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(round(sum_over_ranks(launches, dist))) if dist else int(launches),
        "clocks": clk,
    }
    print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
