#!/usr/bin/env python3
"""Throughput of the force-evaluation hot path (one JSON line on rank 0).

Default workload: HMF model, N = 50,000,000, water-bag initial state
(theta ~ U[-1,1), p ~ U[-1.2,1.2), seed 2), dt = 0.1; one benchmark step is one
integrator step of Sec. 3 (three fused force + kick + drift stages).  Metric:
particle-steps/s on the FP32-sine/FP64-state ("mixed") path, with the FP64 path
and the relative energy errors of both reported beside it.

Other workloads (--workload ring | grav2d) time the all-pairs kernels on the
Ring (N = 131,072, eps = 0.01, dt = 0.05) and 2D (N = 262,144, eps = 1e-4,
dt = 0.01) systems in pair-interactions/s (3 N^2 per step).

--impl reference times the FP64 CPU oracle on the host cores instead.
Under torchrun (N > 1 GPUs) every rank runs an independent replica (the systems
are independent; weak scaling) and the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pair-interactions/s & particle-steps/s, mixed vs FP64, at stated energy error"
WORKLOADS = {
    "hmf": dict(model=0, N=50_000_000, eps=0.0, dt=0.1, seed=2, unit="particle-steps/s",
                name="HMF water-bag N=50,000,000 dt=0.1 (fused reduction+kick/drift)"),
    "ring": dict(model=1, N=131_072, eps=0.01, dt=0.05, seed=3, unit="pair-interactions/s",
                 name="Ring N=131,072 eps=0.01 dt=0.05 (all-pairs)"),
    "grav2d": dict(model=2, N=262_144, eps=1e-4, dt=0.01, seed=4, unit="pair-interactions/s",
                   name="2D self-gravitating N=262,144 eps=1e-4 dt=0.01 (all-pairs)"),
    "grav3d": dict(model=3, N=131_072, eps=1e-3, dt=0.01, seed=5, unit="pair-interactions/s",
                   name="3D self-gravitating N=131,072 eps=1e-3 dt=0.01 (all-pairs; not one of the paper's models)"),
    "sheet1d": dict(model=4, N=262_144, eps=0.0, dt=0.01, seed=6, unit="pair-interactions/s",
                    name="1D sheets N=262,144 eps=0 dt=0.01 (all-pairs sign counts; not one of the paper's models)"),
    "adjoint": dict(model=2, N=262_144, eps=1e-4, dt=0.01, seed=4, unit="pair-interactions/s",
                    name="2D N=262,144 eps=1e-4 dt=0.01: gradient of K(T) after 100 steps (forward + "
                         "reversed adjoint, checkpoints every 20 steps)"),
    "ensemble": dict(model=-1, N=0, eps=0.0, dt=0.0, seed=1000, unit="pair-interactions/s",
                     name="ensemble: 128 Ring (eps=0.01, dt=0.05) + 128 2D (eps=1e-4, dt=0.01), "
                          "N log-uniform in [4096, 65536], one persistent launch per stage"),
}
# algorithmic bytes per particle per fused HMF stage: read + write FP64 theta and p
HMF_BYTES_PER_PARTICLE_STAGE = 32
# FP64-pipe operations per particle of the FP64 HMF stage (its bound): the force
# cos(theta) My - sin(theta) Mx (product + FMA), the kick and the drift (2 FMA), the
# table-driven sine and cosine of the new angle (8: exact FMA reduction, r^2, cos r - 1,
# sin r, two FMAs each for the angle addition)
HMF_FP64_OPS_PER_PARTICLE_STAGE = 12
# FP32-pipe operations and SFU operations per pair in the mixed pair kernels
PAIR_OPS = {1: (8, 1), 2: (6, 1), 3: (11, 1), 4: (4, 0)}
# Per force-kernel variant (md_force_kernel): name, FP32 operations and SFU operations
# per evaluated pair term, and whether each unordered pair is evaluated once.
#   one-sided Ring: S and sin(d/2) (2 FMA + 2 MUL), dd (FMA), y^2, S y, acc (FMA) -> 8
#   tensor-core Ring: S and sin(d/2) on the tensor cores -> 4
#   one-sided 2D: dx, dy, |r|^2 + eps (2 FMA), fx, fy -> 6
#   one-sided 3D: dx, dy, dz, |r|^2 + eps (3 FMA), y^3 (2 MUL), fx, fy, fz -> 11
#   symmetric: + 1 (Ring) / 2 (2D) / 3 (3D) column accumulations per pair term, plus
#   the butterfly adds (1/8 per term for Ring, 1/4 for 2D, 3/4 for 3D at 4 rows/thread)
PAIR_KERNELS = {
    (1, 2): ("streamk_kernel<RingMixed<8,256>>", 8, 1, False),
    (1, 3): ("streamk_kernel<RingTC<4,256>>", 4, 1, False),
    (1, 5): ("sym_kernel<RingTC<4,256>>", 5.125, 1, True),
    (2, 2): ("streamk_kernel<GravMixed<8,256>>", 6, 1, False),
    (2, 4): ("sym_kernel<GravMixed<8,256>>", 8.25, 1, True),
    (3, 2): ("streamk_kernel<Grav3DMixed<4,256>>", 11, 1, False),
    (3, 4): ("sym_kernel<Grav3DMixed<4,256>>", 14.75, 1, True),
    # sheets at eps = 0: difference, two comparisons turned into +-1, accumulate (no SFU)
    (4, 2): ("streamk_kernel<SheetMixed<8,256>>", 4, 0, False),
    (4, 4): ("sym_kernel<SheetMixed<8,256>>", 5.25, 0, True),
}
# FP64 kernels: name, FP64-pipe operations per evaluated pair term (the reciprocal
# square root or reciprocal: FP32 seed on the SFU with integer-pipe conversions, then
# 5 or 3 FP64 operations), whether each unordered pair is evaluated once.
#   Ring: S and sin(d/2) (2 each), dd, rsqrt (5); symmetric: S y^3 (3), row and column
#   adds, butterfly 1/2 -> 15.5; one-sided: S y, y^2, accumulate -> 13
#   2D: dx, dy, s (2), rcp (3); symmetric: 2 products, 2 row and 2 column adds,
#   butterfly 1 -> 14; one-sided: 2 FMA accumulations -> 9
#   3D: dx, dy, dz, s (3), rsqrt (5), y^3 (2); symmetric: 3 products, 3 + 3 adds,
#   butterfly 1.4 -> 23.4; one-sided: 3 FMA accumulations -> 16
PAIR_KERNELS_FP64 = {
    (1, 6): ("sym_kernel<RingF64<4,128>>", 15.5, True),
    (1, 1): ("streamk_kernel<RingF64<2,128>>", 13, False),
    (2, 6): ("sym_kernel<GravF64<4,128>>", 14, True),
    (2, 1): ("streamk_kernel<GravF64<2,128>>", 9, False),
    (3, 6): ("sym_kernel<Grav3DF64<4,128>>", 23.4, True),
    (3, 1): ("streamk_kernel<Grav3DF64<2,128>>", 16, False),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--warmup", type=int, default=None)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="hmf", choices=sorted(WORKLOADS))
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-cores", type=int, default=0,
                    help="processes of the oracle legs (0 = every core of this process's affinity set)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--n", "--particles", dest="n", type=int, default=None,
                    help="override N (profiling runs on smaller cases); --particles under torchrun, whose "
                         "own parser takes --n for one of its options")
    ap.add_argument("--tune", action="append", default=[], help="md_set_tuning key=value (repeatable)")
    ap.add_argument("--repeats", type=int, default=5,
                    help="timed regions of K steps each; value is the median")
    ap.add_argument("--shards", type=int, default=0,
                    help="time the row-shard path instead: the system split among this many shard "
                         "contexts on this GPU, md_shard_step with an exchange after every stage")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the short Ring, 2D and ensemble runs added to the default (HMF) line")
    a = ap.parse_args()
    dflt = {"hmf": (1000, 10), "ring": (20, 3), "grav2d": (10, 3), "grav3d": (20, 3), "sheet1d": (20, 3), "ensemble": (20, 3),
            "adjoint": (1, 3)}[a.workload]
    if a.steps is None:
        a.steps = dflt[0]
    if a.warmup is None:
        a.warmup = dflt[1]
    return a


# ------------------------------------------------------------ utilities ---

def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def src_digest(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, files, units: float):
    """DRAM bytes per launch from the committed ncu summary, scaled to `units`
    (particles), or None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh).get(kernel)
    except Exception:
        return None
    if not rec or rec.get("src_digest") != src_digest(files):
        return None
    return rec["dram_bytes_per_launch"] * units / rec["units"]


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [l.split(",") for l in self.tmp.read().splitlines() if l.count(",") >= 8]
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(float(r[1]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        seen = set()
        for r in rows:
            for k, nm in enumerate(names):
                if "Active" in r[5 + k] and "Not" not in r[5 + k]:
                    seen.add(nm)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(rows[0][2]), "reasons": sorted(seen),
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].strip()
                                                          not in ("", "[N/A]"))}


def device_uuid(dev):
    import torch

    try:
        u = torch.cuda.get_device_properties(dev).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        return None


# ------------------------------------------------------------ oracle legs -

def _oracle_part(w, part: int, parts: int, n: int, steps: int, warmup: int, barrier=None, out=None):
    """One share of the oracle leg, run in this process or in a spawned one.
    HMF: an n-particle water-bag drawn from the workload's seed (every share runs
    its own replica), `steps` integrator steps in one call.  Ring/2D: every
    parts-th of n sampled rows, 3 force evaluations per step against all N
    partners (direct pair sums).  Timed on CLOCK_MONOTONIC from a barrier shared
    by all shares; returns (or puts) (units, t_start, t_end)."""
    import numpy as np

    import oracle as ora
    from paper_1212_0262_gb300 import inputs

    model, N = w["model"], w["N"]
    if model == 0:
        q, p = inputs.waterbag(n, w["seed"])
        if warmup:
            q, p = ora.step(0, q, p, 0.0, w["dt"], warmup)
        units = n * steps

        def work():
            ora.step(0, q, p, 0.0, w["dt"], steps)
    else:
        q, _ = inputs.default_state(model, N, w["seed"])
        rows = np.linspace(0, N - 1, n).astype(np.int64)[part::parts]
        for _ in range(3 * warmup):
            ora.force_rows(model, q, rows, w["eps"])
        units = 3 * len(rows) * N * steps

        def work():
            for _ in range(3 * steps):
                ora.force_rows(model, q, rows, w["eps"])
    if barrier is not None:
        barrier.wait(timeout=600)
    t0 = time.monotonic()
    work()
    t1 = time.monotonic()
    if out is None:
        return units, t0, t1
    out.put((units, t0, t1))
    return None


def host_cores() -> int:
    """Cores this process may run on (its CPU affinity set)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _spawn_parts(target, part_args):
    """Run target(*args, barrier, out) once per entry of part_args in spawned processes
    (no CUDA state is inherited) and return their (units, t_start, t_end) reports."""
    import multiprocessing as mp
    import queue

    n = len(part_args)
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(n), ctx.Queue()
    procs = [ctx.Process(target=target, args=tuple(a) + (barrier, out), daemon=True) for a in part_args]
    for pr in procs:
        pr.start()
    res = []
    t_end = time.monotonic() + 900
    try:
        while len(res) < n:
            try:
                res.append(out.get(timeout=1.0))
            except queue.Empty:
                failed = [pr.exitcode for pr in procs if pr.exitcode not in (None, 0)]
                if failed or time.monotonic() > t_end:
                    raise RuntimeError(f"oracle leg: worker processes failed (exit codes {failed})")
    finally:
        for pr in procs:
            pr.join(timeout=30)
            if pr.is_alive():
                pr.terminate()
    return res


def oracle_steps(w, n: int, steps: int, warmup: int = 0, cores: int = 1):
    """Run the FP64 CPU oracle, as it stands, on a sample of the workload over
    `cores` processes and return (units processed in the timed steps, wall
    seconds, description)."""
    model, N = w["model"], w["N"]
    if cores <= 1:
        units, t0, t1 = _oracle_part(w, 0, 1, n, steps, warmup)
        el = t1 - t0
    else:
        res = _spawn_parts(_oracle_part, [(w, k, cores, n, steps, warmup) for k in range(cores)])
        units = sum(r[0] for r in res)
        el = max(r[2] for r in res) - min(r[1] for r in res)
    if model == 0:
        who = f"{cores} processes, each " if cores > 1 else ""
        desc = f"{who}{n}-particle HMF water-bag (seed {w['seed']}), {steps} oracle steps in one call"
    else:
        over = f" split over {cores} processes" if cores > 1 else ""
        desc = (f"{n} of {N} rows{over} x {N} partners, 3 force evaluations per step, "
                f"{steps} steps (direct pair sums)")
    return units, el, desc


def _oracle_grad_part(w, n: int, nsteps: int, grads: int, barrier=None, out=None):
    """`grads` oracle gradients of K(T) after nsteps steps on an n-particle system
    of the workload's recipe (each process its own replica); pair interactions
    counted as the GPU leg counts them, n^2 (6 nsteps + 1) per gradient."""
    import oracle as ora
    from paper_1212_0262_gb300 import inputs

    q, p = inputs.default_state(w["model"], n, w["seed"])
    ora.grad(w["model"], q, p, w["eps"], w["dt"], 1)
    if barrier is not None:
        barrier.wait(timeout=600)
    t0 = time.monotonic()
    for _ in range(grads):
        ora.grad(w["model"], q, p, w["eps"], w["dt"], nsteps)
    t1 = time.monotonic()
    units = float(n) * n * (6 * nsteps + 1) * grads
    if out is None:
        return units, t0, t1
    out.put((units, t0, t1))
    return None


def oracle_grad(w, seconds: float, grads: int, nsteps: int = 100, cores: int = 1):
    """The oracle's discrete adjoint on an n-particle sample, n sized so that `grads`
    gradients take about `seconds` per process: (units, wall seconds, description)."""
    u0, t0, t1 = _oracle_grad_part(w, 64, nsteps, 1)
    per_unit = (t1 - t0) / u0
    n = int((seconds / grads / per_unit / (6 * nsteps + 1)) ** 0.5)
    n = max(64, min(w["N"], n))
    if cores <= 1:
        units, a, b = _oracle_grad_part(w, n, nsteps, grads)
        el = b - a
    else:
        res = _spawn_parts(_oracle_grad_part, [(w, n, nsteps, grads)] * cores)
        units = sum(r[0] for r in res)
        el = max(r[2] for r in res) - min(r[1] for r in res)
    who = f"{cores} processes, each " if cores > 1 else ""
    return units, el, (f"{who}{grads} oracle gradient(s) of K(T) after {nsteps} steps on a system of {n} particles "
                       f"of the same recipe (forward pass storing every kick position, reversed "
                       f"adjoint pass; n^2 (6 nsteps + 1) pair interactions each)")


def oracle_sample_size(w, seconds: float, steps: int, cores: int = 1) -> int:
    """Sample size so that `steps` oracle steps over `cores` processes take about
    `seconds` here (HMF: the replica size; Ring/2D: the rows over all processes)."""
    model, N = w["model"], w["N"]
    n0 = 20000 if model == 0 else 2
    units, el, _ = oracle_steps(w, n0, 1)
    per_unit = el / units
    per_step_units = seconds / steps / per_unit
    if model == 0:
        # replicas of at most 2e6 particles each when several processes run
        return max(1000, min(N, int(per_step_units), 2_000_000 if cores > 1 else N))
    return max(cores, min(N, int(per_step_units / (3 * N)) * cores))


def ensemble_oracle(seconds: float, steps: int, warmup: int, cores: int):
    """The oracle on one Ring and one 2D member of the ensemble (the first of each
    half), about `seconds` each: (units, seconds, description)."""
    models, Ns, eps, dts, seeds = ensemble_spec()
    units = el = 0.0
    parts = []
    for s in (0, len(Ns) // 2):
        ws_ = dict(model=models[s], N=int(Ns[s]), eps=eps[s], dt=dts[s], seed=seeds[s])
        n = oracle_sample_size(ws_, seconds, steps + warmup, cores)
        u_, e_, smp = oracle_steps(ws_, n, steps, warmup, cores)
        units += u_
        el += e_
        parts.append(f"system {s} ({'Ring' if models[s] == 1 else '2D'}, N={Ns[s]}): {smp}")
    return units, el, "; ".join(parts)


def run_reference(args, w):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    K, W = args.steps, args.warmup
    cores = args.cpu_cores or host_cores()
    if w["model"] == -1:
        units, el, sample = ensemble_oracle(30.0, K, W, cores)
        rate = units / el
    elif args.workload == "adjoint":
        units, el, sample = oracle_grad(w, 60.0 / max(1, K + W) * K, K, cores=cores)
        rate = units / el
    else:
        n = oracle_sample_size(w, 60.0, K + W, cores)
        units, el, sample = oracle_steps(w, n, K, W, cores)
        rate = units / el
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": w["unit"], "n_gpus": args.gpus,
        "steps": K, "warmup": W, "ms_per_step": 1e3 * el / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"]},
        "cpu_baseline": {"kind": "oracle", "cores": cores, "sample": sample, "value": rate, "unit": w["unit"]},
        "e2e": {"value": rate, "unit": w["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ our path ----

def pair_timed_steps(lib, h, stream, flush, K):
    """K integrator steps of a pair model as md_stage calls (the stage list of
    md_step(K): 3K fused stages and the closing kick), L2 flushed before every step;
    returns (total ms, per-stage ms) from CUDA events on the stream."""
    import torch

    from paper_1212_0262_gb300 import binding
    from paper_1212_0262_gb300.system import stage_schedule

    sched = stage_schedule(K)
    elapsed_ms, stage_ms = 0.0, []
    for s in range(K):
        with torch.cuda.stream(stream):
            flush.fill_(float(s))
        sc = sched[3 * s:3 * s + 3] + ([sched[-1]] if s == K - 1 else [])
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(len(sc) + 1)]
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            for k, (b, d) in enumerate(sc):
                binding.check(lib.md_stage(h, b, d), h)
                ev[k + 1].record(stream)
        ev[-1].synchronize()
        ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(len(sc))]
        stage_ms += ms
        elapsed_ms += sum(ms)
    return elapsed_ms, stage_ms


def pipe_rates():
    import numpy as np

    from paper_1212_0262_gb300 import binding

    rates = np.zeros(19)
    binding.load_peaks().mdp_pipe_rates(rates.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 19)
    return rates


def pair_roofline(workload, model, N, kcode, prec, stage_ms, clocks, tuned):
    """Roofline object of a pair-model run: algorithmic pair terms per stage over the
    average stage time, against the pipe-bound rate of the kernel that ran (FP32 and
    SFU operations per term for the FP32 kernels, FP64-pipe operations for the FP64
    ones) at the SM clock sampled during the run; also the fraction at the maximum
    clock."""
    rates = pipe_rates()
    avg_ms = sum(stage_ms) / len(stage_ms)
    nsm = rates[0]
    fp32_rate = max(rates[1], rates[3])  # FP32 FMA ops per SM per clock
    sfu_rate = rates[5] if model in (1, 3) else rates[7]  # rsqrt (Ring, 3D) or rcp (2D)
    kname, fops, sops, sym = PAIR_KERNELS.get((model, kcode), (f"pair kernel {kcode}",) + PAIR_OPS[model] + (False,))
    pairs_per_clk = min(fp32_rate / fops, sfu_rate / sops) if sops else fp32_rate / fops
    f64 = PAIR_KERNELS_FP64.get((model, kcode)) if prec == "fp64" else None
    if f64:  # FP64 kernels: bound by the FP64 pipe (measured DFMA rate)
        kname, dops, sym = f64
        pairs_per_clk = rates[13] / dops
    if prec == "fp64" and not f64:
        return None  # FP64 sheets: sign counting, no stated pipe bound
    mhz = clocks.get("sm_mhz") or rates[2]
    max_mhz = clocks.get("sm_max_mhz") or rates[2]
    peak = nsm * pairs_per_clk * mhz * 1e6
    # algorithmic pair terms per force pass: N^2 ordered pairs, or N (N - 1) / 2
    # unordered pairs when each is evaluated once
    terms = N * (N - 1) / 2 if sym else float(N) * N
    achieved = terms / (avg_ms * 1e-3)
    # DRAM bytes per stage (pair and finish kernels) of the default symmetric FP32
    # kernels, from the committed ncu record when the sources are unchanged
    traffic = None
    if prec == "mixed" and (model, kcode) in ((1, 5), (2, 4)) and not tuned:
        traffic = recorded_traffic(f"{workload}_stage_sym_mixed",
                                   ["paper_1212_0262_gb300/csrc/sym.cu",
                                    "paper_1212_0262_gb300/csrc/pairs_impl.cuh",
                                    "paper_1212_0262_gb300/csrc/md_internal.cuh"], float(N) * N)
    return {"bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "unordered pair terms/s" if sym else "pair-interactions/s",
            "frac": achieved / peak, "frac_at_max_clock": achieved / (peak * max_mhz / mhz), "traffic": traffic,
            "kernel": f"{kname}, {prec}",
            "peak_derivation": ({"sms": nsm, "fp64_ops_per_sm_clk": rates[13], "fp64_ops_per_pair": f64[1],
                                 "sm_mhz": mhz, "sm_max_mhz": max_mhz} if f64 else
                                {"sms": nsm, "fp32_ops_per_sm_clk": fp32_rate,
                                 "sfu_ops_per_sm_clk": sfu_rate, "fp32_ops_per_pair": fops,
                                 "sfu_ops_per_pair": sops, "sm_mhz": mhz, "sm_max_mhz": max_mhz}),
            "pair_terms_per_launch": terms, "avg_launch_ms": avg_ms}


def hmf_fp64_roofline(particle_steps_per_s, rates, clocks):
    """Roofline object of the FP64 HMF path, which the FP64 pipe bounds: 3 stages per step
    of HMF_FP64_OPS_PER_PARTICLE_STAGE FP64 operations per particle, against the SM count
    times the measured FP64 FMA rate per SM per clock (mdp_pipe_rates) at the SM clock
    sampled during the timed region (the rate's own clock without one); also the
    fraction at the maximum clock."""
    nsm, dfma = float(rates[0]), float(rates[13])
    mhz = clocks.get("sm_mhz") or float(rates[14])
    max_mhz = clocks.get("sm_max_mhz") or mhz
    achieved = particle_steps_per_s * 3 * HMF_FP64_OPS_PER_PARTICLE_STAGE
    peak = nsm * dfma * mhz * 1e6
    return {"bound": "alu", "pipe": "fp64", "achieved": achieved, "peak": peak, "unit": "FP64 op/s",
            "frac": achieved / peak, "frac_at_max_clock": achieved / (peak * max_mhz / mhz), "traffic": None,
            "kernel": "hmf_stage_kernel<fp64, kick+drift>",
            "peak_derivation": {"sms": nsm, "fp64_ops_per_sm_clk": dfma,
                                "fp64_ops_per_particle_stage": HMF_FP64_OPS_PER_PARTICLE_STAGE,
                                "sm_mhz": mhz, "sm_max_mhz": max_mhz}}


def secondary_pair(workload, K, W, local, prec="mixed"):
    """A short run of one pair configuration in the default kernels of `prec` (its own
    system, L2 flush, clock record and energy errors after the W warm-up steps and
    after all W + K steps), for the default line."""
    import torch

    from paper_1212_0262_gb300 import System, binding

    w = WORKLOADS[workload]
    model, N = w["model"], w["N"]
    stream = torch.cuda.Stream()
    lib = binding.load()
    with System(model, N, w["eps"], w["dt"], w["seed"], precision=prec) as s:
        s.set_stream(stream)
        e0 = sum(s.energy())
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
        if W:
            pair_timed_steps(lib, s._h, stream, flush, W)
        torch.cuda.synchronize()
        e_w = sum(s.energy())
        sampler = ClockSampler(device_uuid(local))
        l0 = s.launch_count
        elapsed_ms, stage_ms = pair_timed_steps(lib, s._h, stream, flush, K)
        torch.cuda.synchronize()
        launches = s.launch_count - l0
        clocks = sampler.stop()
        e1 = sum(s.energy())
        kcode = s.force_kernel
        del flush
    return {"workload": w["name"], "value": 3.0 * N * N * K / (elapsed_ms * 1e-3), "unit": w["unit"],
            "steps": K, "warmup": W, "ms_per_step": elapsed_ms / K, "precision": prec,
            "rel_energy_error": abs((e1 - e0) / e0), "energy_error_steps": W + K,
            "rel_energy_error_after_warmup": abs((e_w - e0) / e0),
            "roofline": pair_roofline(workload, model, N, kcode, prec, stage_ms, clocks, []),
            "gpu_launches": launches, "clocks": clocks, "l2": "flushed (256 MB write) before every timed step"}


def run_ours(args, w):
    import numpy as np
    import torch

    from paper_1212_0262_gb300 import System, binding

    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    model, N, K, W = w["model"], w["N"], args.steps, args.warmup
    sysm = System(model, N, w["eps"], w["dt"], w["seed"] + 1000 * rank, precision=args.prec)
    sysm.set_stream(stream)
    for kv in args.tune:
        k, v = kv.split("=")
        sysm.set_tuning(k, int(v))
    e0 = sum(sysm.energy())

    lib = binding.load()
    h = sysm._h
    flush = None
    if model != 0:
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    if W:
        if model == 0:
            # the timed region is md_step: capture its step graphs (both ping-pong
            # parities) before timing
            sysm.step(max(W, 9))
            sysm.step(max(W, 9) + 1)
        else:
            pair_timed_steps(lib, h, stream, flush, W)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()

    sampler = ClockSampler(device_uuid(local))
    launches0 = sysm.launch_count
    stage_ms = []
    repeats_ms = None
    if model == 0:
        # md_step(K) as a user calls it: 3K fused kick-drift stages (replayed from captured
        # graphs after the first step) and the closing kick, timed with events on its
        # stream; `repeats` such regions, each bracketed by a synchronize (and a barrier
        # under torchrun), the slowest rank's time per region, the median reported
        repeats_ms = []
        for _ in range(max(1, args.repeats)):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            torch.cuda.synchronize()
            if ws > 1:
                torch.distributed.barrier()
            with torch.cuda.stream(stream):
                ev[0].record(stream)
                sysm.step(K)
                ev[1].record(stream)
            ev[1].synchronize()
            t = torch.tensor([ev[0].elapsed_time(ev[1])], dtype=torch.float64, device=dev)
            if ws > 1:
                torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            repeats_ms.append(float(t.item()))
        elapsed_ms = sorted(repeats_ms)[len(repeats_ms) // 2]
    else:
        # compute-bound kernels on L2-sized inputs: flush L2 between timed steps; `repeats`
        # timed regions of K steps, the median one reported (with its per-stage times)
        repeats_ms = []
        runs = []
        for _ in range(max(1, args.repeats)):
            torch.cuda.synchronize()
            if ws > 1:
                torch.distributed.barrier()
            el, st_ms = pair_timed_steps(lib, h, stream, flush, K)
            t = torch.tensor([el], dtype=torch.float64, device=dev)
            if ws > 1:
                torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            runs.append((float(t.item()), st_ms))
            repeats_ms.append(float(t.item()))
        elapsed_ms, stage_ms = sorted(runs, key=lambda x: x[0])[len(runs) // 2]
    torch.cuda.synchronize()
    launches = (sysm.launch_count - launches0) // len(repeats_ms)
    clocks = sampler.stop()
    torch.cuda.synchronize()
    t_en = time.perf_counter()
    e1 = sum(sysm.energy())
    energy_ms = 1e3 * (time.perf_counter() - t_en)
    de_mixed = abs((e1 - e0) / e0)

    if model == 0:
        units_per_step = N
        value = ws * N * K / (elapsed_ms * 1e-3)
        # algorithmic bytes of the timed region: 3K kick-drift stages (FP64 theta and p read
        # and written, 32 B per particle) and the closing kick (theta and p read, p written:
        # 24 B), over the region's event time (launch gaps included)
        n_launch = 3 * K + 1
        region_bytes = float(N) * (HMF_BYTES_PER_PARTICLE_STAGE * 3 * K + 24)
        avg_ms = elapsed_ms / n_launch
        peaks, src = measured_peaks()
        achieved = region_bytes / (elapsed_ms * 1e-3) / 1e9
        traffic = recorded_traffic("hmf_stage_mixed", ["paper_1212_0262_gb300/csrc/hmf.cu",
                                                       "paper_1212_0262_gb300/csrc/md_internal.cuh"], N)
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                    "kernel": f"hmf_stage_kernel<{'mixed' if args.prec == 'mixed' else 'fp64'}, kick+drift>",
                    "algorithmic_bytes_per_launch": HMF_BYTES_PER_PARTICLE_STAGE * N,
                    "timed_region_bytes": region_bytes, "avg_launch_ms": avg_ms, "launches": n_launch,
                    "timing": "CUDA events around md_step(K) on its stream",
                    "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)"}
        if args.prec == "fp64":
            # the FP64 stage is bound by the FP64 pipe, not by HBM: that roofline, with the
            # HBM figures beside it (a failure here leaves the HBM object and says why)
            try:
                hbm = roofline
                roofline = hmf_fp64_roofline(N * K / (elapsed_ms * 1e-3), pipe_rates(), clocks)
                roofline.update({"hbm": {k: hbm[k] for k in ("achieved", "peak", "unit", "frac")},
                                 "avg_launch_ms": avg_ms, "launches": n_launch, "timing": hbm["timing"]})
            except Exception as e:  # noqa: BLE001 -- the line is printed either way
                roofline = hbm
                roofline["fp64_pipe_error"] = repr(e)
    else:
        units_per_step = 3 * N * N
        value = ws * 3 * N * N * K / (elapsed_ms * 1e-3)
        roofline = pair_roofline(args.workload, model, N, sysm.force_kernel, args.prec, stage_ms, clocks, args.tune)

    # FP64 path on the same workload (few steps) and the matching mixed energy error
    extra = {}
    # the FP64 observables at an observation point (outside the timed steps): K and the
    # potential, an O(N) pass for HMF and the i<j pair sum for the pair models
    npairs = N * (N - 1) / 2
    extra["energy_pass"] = {"ms": energy_ms, "note": "md_energy, synchronous, after the timed steps"}
    if model != 0:
        extra["energy_pass"].update({"pairs": npairs, "pairs_per_s": npairs / (energy_ms * 1e-3)})
    if not args.no_fp64 and rank == 0:
        # HMF: 1 + 999 steps = T = 100 at dt = 0.1, the time the HMF configuration states
        # its energy error at; the pair models: 1 + 2 steps
        ksh = 999 if model == 0 else 2
        res = {}
        for prec in ("fp64", "mixed"):
            with System(model, N, w["eps"], w["dt"], w["seed"], precision=prec) as s2:
                s2.set_stream(stream)
                for kv in args.tune:
                    k, v = kv.split("=")
                    s2.set_tuning(k, int(v))
                e_a = sum(s2.energy())
                s2.step(1)
                torch.cuda.synchronize()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                s2.step(ksh)
                b.record(stream)
                b.synchronize()
                ms = a.elapsed_time(b)
                e_b = sum(s2.energy())
                units = N * ksh if model == 0 else 3 * N * N * ksh
                res[prec] = {"value": units / (ms * 1e-3), "ms_per_step": ms / ksh,
                             "rel_energy_error": abs((e_b - e_a) / e_a), "steps": ksh + 1}
        extra["fp64_path"] = res["fp64"]
        if model == 0:  # its FP64-pipe roofline at the clock sampled in the timed region above
            try:
                extra["fp64_path"]["roofline"] = hmf_fp64_roofline(res["fp64"]["value"], pipe_rates(), clocks)
            except Exception as e:  # noqa: BLE001 -- the line is printed either way
                extra["fp64_path"]["roofline"] = {"error": repr(e)}
        extra["mixed_path_long_run"] = res["mixed"]
        T = res["mixed"]["steps"] * w["dt"]
        extra["energy_error"] = {"mixed_after_%d_steps" % (res["mixed"]["steps"]): res["mixed"]["rel_energy_error"],
                                 "fp64_after_%d_steps" % (res["fp64"]["steps"]): res["fp64"]["rel_energy_error"],
                                 "T": T, "mixed_timed_run": de_mixed,
                                 "timed_run_steps": W + K * (len(repeats_ms) if repeats_ms else 1)}

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if rank == 0 and not args.no_e2e:
        n = sysm.dim * N
        qh = torch.empty(n, dtype=torch.float64, pin_memory=True)
        ph = torch.empty(n, dtype=torch.float64, pin_memory=True)
        sysm.get_state_device  # noqa: B018  (API presence)
        qn, pn = qh.numpy(), ph.numpy()
        lib.md_get_state(h, ctypes.c_void_p(qn.ctypes.data), ctypes.c_void_p(pn.ctypes.data))
        ke = K  # the timed step count (after md_set_state the first step also primes the force)
        runs = []  # three timed end-to-end regions, the median one reported
        for _ in range(3):
            torch.cuda.synchronize()
            tp = [time.perf_counter()]
            binding.check(lib.md_set_state(h, ctypes.c_void_p(qn.ctypes.data), ctypes.c_void_p(pn.ctypes.data)), h)
            tp.append(time.perf_counter())
            binding.check(lib.md_step(h, ke), h)
            binding.check(lib.md_synchronize(h), h)
            tp.append(time.perf_counter())
            kk, vv = ctypes.c_double(), ctypes.c_double()
            binding.check(lib.md_energy(h, ctypes.byref(kk), ctypes.byref(vv)), h) if model == 0 else None
            tp.append(time.perf_counter())
            binding.check(lib.md_get_state(h, ctypes.c_void_p(qn.ctypes.data), ctypes.c_void_p(pn.ctypes.data)), h)
            tp.append(time.perf_counter())
            runs.append(tp)
        tp = sorted(runs, key=lambda t: t[-1] - t[0])[1]
        el = tp[-1] - tp[0]
        e2e = {"value": (N * ke if model == 0 else 3 * N * N * ke) / el, "unit": w["unit"],
               "h2d_bytes_per_step": 2 * 8 * n / ke, "d2h_bytes_per_step": (2 * 8 * n + (16 if model == 0 else 0)) / ke,
               "steps": ke, "note": "md_set_state(host) + md_step + " + ("md_energy + " if model == 0 else "")
               + "md_get_state(host), wall clock" + ("" if model == 0 else
               "; the O(N^2) potential is an observation-point pass, timed as energy_pass"),
               "parts_ms": {k: 1e3 * (tp[i + 1] - tp[i]) for i, k in
                            enumerate(("set_state", "step", "energy", "get_state"))},
               "runs_s": [t[-1] - t[0] for t in runs], "reported": "median of 3 timed regions"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        ksteps = 4 if model == 0 else 1
        cores = args.cpu_cores or host_cores()
        n1 = oracle_sample_size(w, 5.0, ksteps)
        u1, e1, s1 = oracle_steps(w, n1, ksteps)
        n = oracle_sample_size(w, 10.0, ksteps, cores)
        if model == 0:  # capped replicas: more steps instead, about the same seconds
            ksteps = max(ksteps, int(round(ksteps * oracle_sample_size(w, 10.0, ksteps) / n)))
        units, el, sample = oracle_steps(w, n, ksteps, 0, cores)
        cpu = {"value": units / el, "unit": w["unit"], "cores": cores, "kind": "oracle", "sample": sample,
               "seconds": el, "single_core": {"value": u1 / e1, "sample": s1, "seconds": e1}}

    # the other configurations, each a short driver-clocked run with its own clock
    # record and roofline: Ring (N = 131,072), 2D forward (N = 262,144) and the ensemble
    secondary = None
    if rank == 0 and model == 0 and not args.no_secondary and not args.n:
        sysm.close()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        # 20 / 10 / 10 steps: the closing kick-only stage of each timed call (a force
        # pass not counted in the 3 N^2 per step) stays within 1.6-3% of the time
        secondary = {"ring": secondary_pair("ring", 20, 3, local), "grav2d": secondary_pair("grav2d", 10, 3, local)}
        # the FP64 kernels on the same systems: 1 + 2 steps, so that both precisions state
        # their energy error after the same 3 steps (the mixed runs' warm-up)
        for wl in ("ring", "grav2d"):
            f64 = secondary_pair(wl, 2, 1, local, prec="fp64")
            secondary[wl]["fp64"] = f64
            secondary[wl]["energy_error_3_steps"] = {"mixed": secondary[wl]["rel_energy_error_after_warmup"],
                                                     "fp64": f64["rel_energy_error"]}
        ens, _, _, m = ensemble_measure("mixed", 10, 3, local, repeats=3)
        ens.close()
        m.pop("pairs_per_stage")
        secondary["ensemble"] = dict(workload=WORKLOADS["ensemble"]["name"], unit=WORKLOADS["ensemble"]["unit"],
                                     steps=10, warmup=3, precision="mixed", **m)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": w["unit"], "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": elapsed_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 state / f32 " + ("sin,cos" if model == 0 else "pair arithmetic") if args.prec == "mixed" else "f64",
            "data": "synthetic",
            "config": {"workload": w["name"], "N": N, "eps": w["eps"], "dt": w["dt"], "seed": w["seed"],
                       "precision": args.prec, "parallelism": f"replicas x{ws}", "tuning": args.tune,
                       "l2": "state 800 MB > L2 (no flush needed)" if model == 0 else "L2 flushed (256 MB write) between timed steps"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
            "rel_energy_error": de_mixed,
        }
        if repeats_ms is not None:
            line["repeats_ms"] = repeats_ms
        line.update(extra)
        if secondary is not None:
            line["secondary"] = secondary
        print(json.dumps(line), flush=True)
    sysm.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


def ensemble_spec(nsys=256, seed=1000):
    """Models, sizes, softenings, steps and seeds of the batched-ensemble workload."""
    from paper_1212_0262_gb300 import inputs

    Ns = inputs.ensemble_sizes(nsys, seed)
    models = [1 if s < nsys // 2 else 2 for s in range(nsys)]
    eps = [0.01 if m == 1 else 1e-4 for m in models]
    dts = [0.05 if m == 1 else 0.01 for m in models]
    seeds = [seed + s for s in range(nsys)]
    return models, Ns, eps, dts, seeds


def ensemble_roofline(ens, Ns, models, prec, avg_ms, clocks):
    """Roofline of an ensemble stage: the algorithmic pair terms of all systems over
    the average stage time, against the time-optimal rate for the mix of Ring and 2D
    terms at the sampled SM clock (and at the maximum clock)."""
    import numpy as np

    rates = pipe_rates()
    nsm = rates[0]
    fp32 = max(rates[1], rates[3])
    # kernel form: r = 0 (mixed) evaluates every unordered pair of a system once
    sym = prec == "mixed" and ens.tuning[0] == 0
    kr = PAIR_KERNELS[(1, 5)] if sym else ("batch Ring part", PAIR_OPS[1][0], PAIR_OPS[1][1], False)
    kg = PAIR_KERNELS[(2, 4)] if sym else ("batch 2D part", PAIR_OPS[2][0], PAIR_OPS[2][1], False)
    per_clk_ring = min(fp32 / kr[1], rates[5] / kr[2])
    per_clk_2d = min(fp32 / kg[1], rates[7] / kg[2])
    if sym:
        w_ring = float(sum(n * (n - 1) / 2 for n, m in zip(Ns, models) if m == 1))
        w_2d = float(sum(n * (n - 1) / 2 for n, m in zip(Ns, models) if m == 2))
    else:
        w_ring = float(sum(float(n) * n for n, m in zip(Ns, models) if m == 1))
        w_2d = float(sum(float(n) * n for n, m in zip(Ns, models) if m == 2))
    terms = w_ring + w_2d
    mhz = clocks.get("sm_mhz") or rates[2]
    max_mhz = clocks.get("sm_max_mhz") or rates[2]
    peak = terms / (w_ring / (nsm * per_clk_ring * mhz * 1e6) + w_2d / (nsm * per_clk_2d * mhz * 1e6))
    achieved = terms / (avg_ms * 1e-3)
    return {"bound": "alu", "achieved": achieved, "peak": peak,
            "unit": "unordered pair terms/s" if sym else "pair-interactions/s",
            "frac": achieved / peak, "frac_at_max_clock": achieved / (peak * max_mhz / mhz), "traffic": None,
            "kernel": ("batch_sym_pairs_kernel + batch_sym_finish_kernel (Ring tensor-core + 2D parts)"
                       if sym else "batch_kernel (Ring + 2D parts)"),
            "pair_terms_per_stage": terms, "avg_stage_ms": avg_ms, "sm_mhz": mhz, "sm_max_mhz": max_mhz}


def ensemble_measure(prec, K, W, local, repeats=1, ws=1):
    """The batched-ensemble workload: build, autotune, W warm-up steps, then `repeats`
    timed regions of md_batch_step(K) (CUDA events on the ensemble's stream, each
    bracketed by a synchronize and, under torchrun, a barrier; the slowest rank's time
    per region, the median kept).  Returns (ensemble, spec, stream, measurement dict)."""
    import numpy as np
    import torch

    from paper_1212_0262_gb300 import Ensemble

    stream = torch.cuda.Stream()
    models, Ns, eps, dts, seeds = ensemble_spec()
    ens = Ensemble(models, Ns, eps, dts, seeds, precision=prec)
    ens.set_stream(stream)
    t0 = time.perf_counter()
    tuned_ms = ens.autotune()
    tune_s = time.perf_counter() - t0
    K0, V0 = ens.energy()
    if W:
        ens.step(W)
    pairs_per_stage = float(np.sum(np.asarray(Ns, dtype=np.float64) ** 2))
    sampler = ClockSampler(device_uuid(local))
    l0 = ens.launch_count
    reps = []
    for _ in range(max(1, repeats)):
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ens.step(K)
        b.record(stream)
        b.synchronize()
        t = torch.tensor([a.elapsed_time(b)], dtype=torch.float64, device="cuda")
        if ws > 1:
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        reps.append(float(t.item()))
    launches = (ens.launch_count - l0) // len(reps)
    clocks = sampler.stop()
    ms = sorted(reps)[len(reps) // 2]
    K1, V1 = ens.energy()
    e0, e1 = K0 + V0, K1 + V1
    de = np.abs((e1 - e0) / e0)
    avg_ms = ms / (3 * K + 1)
    m = {"value": ws * 3 * pairs_per_stage * K / (ms * 1e-3), "ms_per_step": ms / K, "repeats_ms": reps,
         "roofline": ensemble_roofline(ens, Ns, models, prec, avg_ms, clocks),
         "autotune": {"seconds": tune_s, "best_force_launch_ms": tuned_ms, "tuning": list(ens.tuning)},
         "rel_energy_error": {"max": float(de.max()), "median": float(np.median(de)),
                              "steps": W + K * len(reps)},
         "gpu_launches": launches, "clocks": clocks, "pairs_per_stage": pairs_per_stage}
    return ens, (models, Ns, eps, dts, seeds), stream, m


def run_ensemble(args, w):
    import ctypes as _c

    import numpy as np
    import torch

    from paper_1212_0262_gb300 import binding

    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    K, W = args.steps, args.warmup
    ens, (models, Ns, eps, dts, seeds), stream, m = ensemble_measure(args.prec, K, W, local, args.repeats, ws)
    pairs_per_stage = m["pairs_per_stage"]

    e2e = None
    if rank == 0 and not args.no_e2e:
        # every system's state from pinned host memory, the steps and every state
        # back, through the public ensemble API (wall clock)
        dims = [2 if mm == 2 else 1 for mm in models]
        sizes = [d * int(n) for d, n in zip(dims, Ns)]
        offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        qh = torch.empty(int(offs[-1]), dtype=torch.float64, pin_memory=True).numpy()
        ph = torch.empty(int(offs[-1]), dtype=torch.float64, pin_memory=True).numpy()
        for k in range(len(Ns)):
            qk, pk = ens.get_state(k)
            qh[offs[k]:offs[k + 1]], ph[offs[k]:offs[k + 1]] = qk, pk
        ke = K
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(len(Ns)):
            ens.set_state(k, qh[offs[k]:offs[k + 1]], ph[offs[k]:offs[k + 1]])
        ens.step(ke)
        for k in range(len(Ns)):
            b_ = binding.load()
            ens._chk(b_.md_batch_get_state(ens._h, k, _c.c_void_p(qh[offs[k]:].ctypes.data),
                                          _c.c_void_p(ph[offs[k]:].ctypes.data)))
        el = time.perf_counter() - t0
        nb = 2 * 8 * float(offs[-1])
        e2e = {"value": 3 * pairs_per_stage * ke / el, "unit": w["unit"], "h2d_bytes_per_step": nb / ke,
               "d2h_bytes_per_step": nb / ke, "steps": ke,
               "note": "md_batch_set_state(host, every system) + md_batch_step + "
                       "md_batch_get_state(host, every system), wall clock"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cores = args.cpu_cores or host_cores()
        units, el, sample = ensemble_oracle(5.0, 1, 0, cores)
        cpu = {"value": units / el, "unit": w["unit"], "cores": cores, "kind": "oracle", "sample": sample,
               "seconds": el}

    if rank == 0:
        line = {
            "metric": METRIC, "value": m["value"], "unit": w["unit"], "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": m["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 state / f32 pair arithmetic" if args.prec == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": w["name"], "systems": len(Ns), "sum_N": int(np.sum(Ns)),
                       "sum_N2": pairs_per_stage, "precision": args.prec,
                       "l2": "state and mirrors of all systems ~180 MB > L2"},
            "roofline": m["roofline"], "repeats_ms": m["repeats_ms"], "autotune": m["autotune"],
            "rel_energy_error": m["rel_energy_error"],
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": m["gpu_launches"], "clocks": m["clocks"],
        }
        print(json.dumps(line), flush=True)
    ens.close()


def run_adjoint(args, w):
    """md_grad on the 2D configuration: `steps` gradient evaluations of K(T) after
    100 integrator steps; pair interactions counted for both passes (3 N^2 per
    forward step, N^2 per reverse stage, 3 nsteps + 1 reverse stages).  The
    mixed gradient's error is stated against the FP64 gradient at N = 16,384."""
    import numpy as np
    import torch

    from paper_1212_0262_gb300 import System, binding

    ws, rank, local = dist_info()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    N, nsteps, K = w["N"], 100, 20
    s = System(2, N, w["eps"], w["dt"], w["seed"], precision=args.prec)
    s.set_stream(stream)
    for kv in args.tune:
        k, v = kv.split("=")
        s.set_tuning(k, int(v))
    for _ in range(args.warmup):
        s.grad(2, 0, 1)
    sampler = ClockSampler(device_uuid(local))
    l0 = s.launch_count
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        val, gq, gp, ge = s.grad(nsteps, 0, K)
    el = (time.perf_counter() - t0) / args.steps
    launches = s.launch_count - l0
    clocks = sampler.stop()
    pairs = float(N) * N * (3 * nsteps + 3 * nsteps + 1)
    # mixed vs FP64 gradient on a smaller system of the same recipe
    n2 = 16384
    out = {}
    for prec in ("fp64", "mixed"):
        with System(2, n2, w["eps"], w["dt"], w["seed"], precision=prec) as s2:
            out[prec] = s2.grad(nsteps, 0, K)
    e2e = None
    if rank == 0 and not args.no_e2e:
        # the state from pinned host memory and the gradient back to host arrays,
        # through the public API (wall clock)
        qh = torch.empty(2 * N, dtype=torch.float64, pin_memory=True).numpy()
        ph = torch.empty(2 * N, dtype=torch.float64, pin_memory=True).numpy()
        qh[:], ph[:] = s.get_state()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        s.set_state(qh, ph)
        s.grad(nsteps, 0, K)
        e_el = time.perf_counter() - t1
        e2e = {"value": pairs / e_el, "unit": w["unit"], "h2d_bytes_per_step": 2 * 8 * 2 * N,
               "d2h_bytes_per_step": 2 * 8 * 2 * N + 16, "steps": 1,
               "note": "md_set_state(host) + md_grad (gradients to host arrays), wall clock"}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cores = args.cpu_cores or host_cores()
        units, c_el, sample = oracle_grad(w, 10.0, 1, nsteps, cores)
        cpu = {"value": units / c_el, "unit": w["unit"], "cores": cores, "kind": "oracle", "sample": sample,
               "seconds": c_el}
    rel = lambda a, b: float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
    err = {"grad_q": rel(out["mixed"][1], out["fp64"][1]), "grad_p": rel(out["mixed"][2], out["fp64"][2]),
           "grad_eps": abs(out["mixed"][3] - out["fp64"][3]) / abs(out["fp64"][3]), "N": n2}
    # roofline by time: the forward stages (unordered pair terms of the symmetric 2D
    # kernel) and the reverse stages (the one-sided reverse kernel: per ordered pair
    # dx, dy, s (2), inv^2, w (2), the (r.w) product (4), f (2), J w (4), df/deps (2) =
    # 19 FP32 operations and one rcp) at their pipe bounds, against the measured time
    roofline = None
    if args.prec == "mixed":
        rates = np.zeros(19)
        binding.load_peaks().mdp_pipe_rates(rates.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 19)
        nsm, fp32 = rates[0], max(rates[1], rates[3])
        mhz = clocks.get("sm_mhz") or rates[2]
        clk = nsm * mhz * 1e6
        fwd_terms = 3 * nsteps * N * (N - 1) / 2
        rev_pairs = (3 * nsteps + 1) * float(N) * N
        t_fwd = fwd_terms / (clk * min(fp32 / PAIR_KERNELS[(2, 4)][1], rates[7]))
        t_rev = rev_pairs / (clk * min(fp32 / 19.0, rates[7]))
        roofline = {"bound": "alu", "achieved": (t_fwd + t_rev) / el, "peak": 1.0, "unit": "fraction of the pipe-bound time",
                    "frac": (t_fwd + t_rev) / el, "traffic": None,
                    "kernel": "sym_pairs_kernel<GravMixed> forward + streamk_kernel<GravMixedAdj> reverse",
                    "ideal_seconds": {"forward": t_fwd, "reverse": t_rev}, "sm_mhz": mhz}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": pairs / el, "unit": w["unit"], "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 state / f32 pair arithmetic" if args.prec == "mixed" else "f64",
            "data": "synthetic", "config": {"workload": w["name"], "precision": args.prec, "N": N,
                                            "nsteps": nsteps, "checkpoint_every": K},
            "gradient_seconds": el, "value_K_T": val, "grad_eps": ge,
            "mixed_vs_fp64_gradient_rel_error": err, "gpu_launches": launches, "clocks": clocks,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e}), flush=True)
    s.close()


def run_shards(args, w):
    """The row-shard path (md_shard_*) on one GPU: the workload's system split among
    `--shards` contexts, K steps of md_shard_step (every stage of every rank, then the
    exchange of every rank's segment), wall-clock timed between device synchronizes.
    Reports the throughput and the exchanged bytes per step beside the whole-system
    one-sided kernel timed the same way."""
    import torch

    from paper_1212_0262_gb300 import ShardGroup, System

    model, N, K, W, P = w["model"], w["N"], args.steps, args.warmup, args.shards
    units = N if model == 0 else 3.0 * N * N

    def timed(step):
        step(W)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(K)
        torch.cuda.synchronize()
        return 1e3 * (time.perf_counter() - t0)

    sampler = ClockSampler(device_uuid(0))
    with ShardGroup(model, N, w["eps"], w["dt"], w["seed"], P, precision=args.prec) as g:
        ms = timed(g.step)
        seg = [g.buffer(r)[2] for r in range(P)]
    clocks = sampler.stop()
    with System(model, N, w["eps"], w["dt"], w["seed"], precision=args.prec) as s:
        if model != 0:
            s.set_tuning("symmetric", 0)  # every ordered pair, as the shards
        ms_whole = timed(s.step)
    # every stage copies each rank's segment into the P - 1 other buffers
    xbytes = 3 * (P - 1) * sum(seg)
    print(json.dumps({
        "metric": METRIC, "value": units * K / (ms * 1e-3), "unit": w["unit"], "n_gpus": 1, "steps": K,
        "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f64" if args.prec == "fp64" else "f64 state / f32 " + ("sin,cos" if model == 0 else "pair arithmetic"),
        "data": "synthetic",
        "config": {"workload": w["name"] + f", split by rows among {P} shard contexts on one GPU",
                   "precision": args.prec, "shards": P, "parallelism": f"row shards x{P} (one GPU)"},
        "whole_system": {"value": units * K / (ms_whole * 1e-3), "ms_per_step": ms_whole / K,
                         "kernel": "one-sided (every ordered pair)" if model else "HMF fused stage"},
        "exchange_bytes_per_step": xbytes, "segment_bytes": seg, "clocks": clocks,
        "note": "wall clock around K steps of md_shard_step (and of md_step for the whole system) between "
                "device synchronizes; on one GPU the shards share the SMs, so this measures the sharded "
                "path's overhead, not multi-GPU scaling"}), flush=True)


def main():
    args = parse()
    if args.shards and args.impl == "ours":
        run_shards(args, dict(WORKLOADS[args.workload], **({"N": args.n} if args.n else {})))
        return
    if args.workload == "ensemble" and args.impl == "ours":
        run_ensemble(args, WORKLOADS["ensemble"])
        return
    w = dict(WORKLOADS[args.workload])
    if args.n:
        w["N"] = args.n
        w["name"] = w["name"].split(" N=")[0] + f" N={args.n:,} (reduced size)"
    if args.workload == "adjoint" and args.impl == "ours":
        run_adjoint(args, w)
        return
    if args.impl == "reference":
        run_reference(args, w)
        return
    run_ours(args, w)


if __name__ == "__main__":
    main()
