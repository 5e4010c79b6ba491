#!/usr/bin/env python
"""Benchmark of the explicit EBE enthalpy step (tet-element updates/s).

Default workload: ``block_with_cores_220`` -- a 1 m alloy block with 32
seeded spherical steel cores, 220^3 hexes x 6 Kuhn tets = 63,888,000 tets,
10,793,861 nodes, 5% nodal jitter, Robin on the outer faces, FP32 stepping
with FP64 energy bookkeeping, block-partitioned atomic-free scatter.  One
benchmark step is one explicit time step over the whole mesh (all kernels of
the step).  Inputs (~2.7 GB of per-step traffic) are larger than the 129 MB
L2, so no flush is needed between steps.

Prints one JSON line.  Beside the GPU figures it times, on a 1.5M-tet sample
of the same recipe, the FP64 oracle on one host core (``cpu_baseline``) and
the threaded OpenMP baseline in FP32 and FP64 on all host cores
(``cpu_threaded``).  ``--impl reference`` times the FP64 CPU oracle on the
host instead (bounded sample of the same workload recipe).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# DRAM bytes per unit of work of a kernel, from one ncu capture (see the
# matching summary under profiles/); valid while the sources it was taken on
# are unchanged
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.json")
TRAFFIC_SOURCES = ("fem_kernels.cu", "fem_state.cuh", "fem_device.cuh", "fem_internal.h",
                   "fem_plan.cpp", "fem_plan.h")


def sources_digest() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, "paper_1005_3158_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(kernel: str, precision: str, variant: str, n_units: int,
                     scope: str = "single"):
    """ncu DRAM bytes (read + write) per launch of `kernel`, scaled from the
    captured workload to n_units by the units processed; None when no
    capture matches or the sources changed since it was taken.  scope is
    "single" (one mesh) or "batch" (a batch of instances)."""
    try:
        with open(TRAFFIC_FILE) as fh:
            entries = json.load(fh)["entries"]
    except (OSError, ValueError, KeyError):
        return None
    digest = sources_digest()
    for e in entries:
        if (e["kernel"], e["precision"], e["variant"]) == (kernel, precision, variant) \
                and e.get("scope", "single") == scope and e["sources_sha256"] == digest:
            per_unit = (e["dram_read_bytes"] + e["dram_write_bytes"]) / e["units"]
            return int(round(per_unit * n_units))
    return None


def max_over_ranks(x: float, world: int, device="cpu") -> float:
    """Max of x over the ranks of the default process group (x for one rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, steps: int, world: int, seconds: float) -> float:
    """Whole-job units per second: every rank processes units_per_rank per
    step (weak scaling), the job takes the slowest rank's time."""
    return units_per_rank * steps * world / seconds


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=None,
                    help="default block_with_cores_220 (or the one --config names)")
    ap.add_argument("--config", type=int, default=0, choices=[0, 1, 2, 3, 4, 5],
                    help="1: unit_cube_20 FP64 (parity case), 2: flanged_casting, "
                         "3: block_with_cores_220 (the default), 4: batched_castings_256, "
                         "5: surrogate_flanged (learned 16-step surrogate vs plain FP32)")
    ap.add_argument("--n-eval", type=int, default=2,
                    help="surrogate workload: unseen 2M-tet castings evaluated (of 10)")
    ap.add_argument("--judge-every", type=int, default=8)
    ap.add_argument("--tol", type=float, default=2.0)
    ap.add_argument("--params", default="")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--variant", default="block", choices=["block", "atomic", "colored"])
    ap.add_argument("--physics", default="const", choices=["const", "kt", "apparent"],
                    help="const: constant k, enthalpy (default); kt: temperature-dependent "
                         "conductivity tables; apparent: the apparent-capacity formulation")
    ap.add_argument("--reorder", type=int, default=1)
    ap.add_argument("--block-elems", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--profile-steps", type=int, default=20)
    ap.add_argument("--autotune", default="",
                    help="comma list of candidate partitions, block_elems or "
                         "block_elems x threads (e.g. 1024,2048,2048x1024): "
                         "fem_autotune keeps the fastest before timing")
    ap.add_argument("--autotune-steps", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=200, help="0 = same as --steps")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-threaded", action="store_true")
    ap.add_argument("--cpu-threaded-seconds", type=float, default=4.0)
    ap.add_argument("--no-sequential", action="store_true",
                    help="batched workload: skip the instance-by-instance comparison")
    a = ap.parse_args()
    named = {1: "unit_cube_20", 2: "flanged_casting", 3: "block_with_cores_220",
             4: "batched_castings_256", 5: "surrogate_flanged"}
    if a.workload is None:
        a.workload = named.get(a.config, "block_with_cores_220")
    if a.config == 1 and "--precision" not in sys.argv:
        a.precision = "fp64"
    return a


def autotune(m, spec: str, steps: int, dt: float):
    """fem_autotune over the --autotune candidates; returns the config record."""
    be, th = [], []
    for c in spec.split(","):
        x = c.strip().lower().split("x")
        be.append(int(x[0]))
        th.append(int(x[1]) if len(x) > 1 else 0)
    t0 = time.perf_counter()
    best, ms = m.autotune(be, th, steps=steps, dt=dt)
    return {"candidates": [f"{b}x{t}" if t else str(b) for b, t in zip(be, th)],
            "ms_per_step": [round(float(v), 5) for v in ms], "chosen": best,
            "steps": steps, "seconds": round(time.perf_counter() - t0, 1)}


def make_problem(name: str):
    from paper_1005_3158_gb300 import meshgen as mg
    if name.startswith("block_with_cores_"):
        return mg.block_with_cores(int(name.rsplit("_", 1)[1]))
    if name.startswith("unit_cube_"):
        return mg.unit_cube(int(name.rsplit("_", 1)[1]))
    if name == "flanged_casting":
        return mg.flanged_casting()
    if name == "flanged_casting_random":
        # the unordered mesh of the ordering comparison: nodes and elements
        # randomly renumbered (seed 1006)
        import numpy as np
        rng = np.random.Generator(np.random.PCG64(1006))
        return mg.permute_elements(mg.permute_nodes(mg.flanged_casting(), rng), rng)
    raise SystemExit(f"unknown workload {name}")


def make_problem_size(name: str) -> int:
    """Number of tets of a named workload (without building it)."""
    if name.startswith("block_with_cores_") or name.startswith("unit_cube_"):
        return 6 * int(name.rsplit("_", 1)[1]) ** 3
    if name.startswith("flanged_casting"):
        return 6 * 70 * 70 * 68
    raise SystemExit(f"unknown workload {name}")


def sample_recipe(name: str, target_tets: float):
    """A smaller problem with the same recipe (for the host-side oracle)."""
    from paper_1005_3158_gb300 import meshgen as mg
    n = max(4, int(round((target_tets / 6.0) ** (1.0 / 3.0))))
    if name.startswith("block_with_cores_"):
        return mg.block_with_cores(n), f"block_with_cores_{n}"
    if name.startswith("unit_cube_"):
        return mg.unit_cube(n), f"unit_cube_{n}"
    return mg.flanged_casting(n, n, n), f"flanged_casting_{n}x{n}x{n}"


def hbm_peak():
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms.  The
    sampler starts before the warm-up steps; when the timed region is short,
    the caller keeps stepping (untimed) after it until the sampler has seen
    `min_s` seconds, so that the record holds several samples under the
    same load."""

    min_s = 1.0

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            self.t0 = time.perf_counter()
        except Exception:
            self.proc = None

    def remaining(self) -> float:
        """Seconds the sampler still wants under load (0 when enough)."""
        if self.proc is None:
            return 0.0
        return max(0.0, self.min_s - (time.perf_counter() - self.t0))

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm), "interval_ms": 50,
                "window": "warm-up, timed region and untimed steps after it (at least "
                          f"{self.min_s:.1f} s under the same step loop)"}


def cpu_baseline(workload: str, seconds: float):
    """The FP64 oracle as it stands, single thread, on a bounded sample of
    the same recipe; returns tet-updates/s."""
    import oracle
    p, name = sample_recipe(workload, 1.5e6)
    o = oracle.OracleProblem(p)
    o.set_temperature(p.T0)
    dt = 0.9 * o.stable_dt()
    o.step(1, dt)
    steps, t0 = 0, time.perf_counter()
    while True:
        o.step(1, dt)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds or steps >= 1000:
            break
    return ({"value": p.n_tets * steps / el, "unit": "tet-updates/s", "cores": 1,
             "kind": "oracle",
             "sample": f"{name} ({p.n_tets} tets), {steps} FP64 steps, {el:.1f} s single-thread"},
            p, name, dt)


def cpu_threaded(p, name: str, dt: float, seconds: float):
    """The threaded CPU baseline (OpenMP, colour-parallel element loop) on
    the oracle's sample, FP32 and FP64, all host cores; tet-updates/s."""
    import cpu_threaded as ct
    out = {}
    for prec in ("fp32", "fp64"):
        with ct.ThreadedBaseline(p, prec) as b:
            b.step(3, dt)
            steps, t0 = 0, time.perf_counter()
            while True:
                b.step(10, dt)
                steps += 10
                el = time.perf_counter() - t0
                if el >= seconds or steps >= 20000:
                    break
            inf = b.info()
        out[prec] = {"value": p.n_tets * steps / el, "unit": "tet-updates/s",
                     "cores": inf["threads"], "kind": "threaded",
                     "sample": f"{name} ({p.n_tets} tets), {steps} {prec.upper()} steps, "
                               f"{el:.1f} s, {inf['colours']} element colours"}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    # each step: one oracle time step on a sample sized so that the whole
    # run stays within about two minutes
    rate_guess = 3.0e7
    full = make_problem_size(args.workload)
    target = min(full, 8.0e6, max(5e4, 120.0 * rate_guess / max(1, args.steps + args.warmup)))
    p, name = sample_recipe(args.workload, target)
    o = oracle.OracleProblem(p)
    o.set_temperature(p.T0)
    dt = 0.9 * o.stable_dt()
    o.step(args.warmup, dt)
    t0 = time.perf_counter()
    o.step(args.steps, dt)
    el = time.perf_counter() - t0
    val = p.n_tets * args.steps / el
    line = {
        "impl": "reference", "metric": "tet-element updates/s", "value": val,
        "unit": "tet-updates/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "sample": name, "sample_tets": p.n_tets,
                   "oracle": "plain FP64 C EBE solver, single thread"},
        "cpu_baseline": {"value": val, "unit": "tet-updates/s", "cores": 1, "kind": "oracle",
                         "sample": f"{name} ({p.n_tets} tets), {args.steps} steps"},
        "e2e": {"value": val, "unit": "tet-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_batch(probs, seconds: float):
    """The FP64 oracle as it stands, single thread, on a bounded subset of
    a batch's instances (the first ones, up to 1.5M tets), each stepped at
    0.9 of its own stable step in turn; returns the cpu_baseline record."""
    import oracle
    sub, tot = [], 0
    for p in probs:
        if sub and tot + p.n_tets > 1.5e6:
            break
        sub.append(p)
        tot += p.n_tets
    os_, dts = [], []
    for p in sub:
        o = oracle.OracleProblem(p)
        o.set_temperature(p.T0)
        os_.append(o)
        dts.append(0.9 * o.stable_dt())
    upd, rounds, t0 = 0.0, 0, time.perf_counter()
    while True:
        for o, d, p in zip(os_, dts, sub):
            o.step(1, d)
            upd += p.n_tets
        rounds += 1
        el = time.perf_counter() - t0
        if el >= seconds or rounds >= 1000:
            break
    return {"value": upd / el, "unit": "tet-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"first {len(sub)} instances of the batch ({tot} tets), {rounds} FP64 "
                      f"steps each at its own dt, {el:.1f} s single-thread"}


def run_batched(args):
    """Batched castings (256 instances, 20k-500k tets each, FP32): one
    fem_advance to a common end time, every instance at 0.9 x its own
    stable step; the instance with the smallest step takes --steps steps.
    Compared with the same steps run instance by instance."""
    import math
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1005_3158_gb300 import fem
    from paper_1005_3158_gb300 import meshgen as mg
    n_inst = int(args.workload.rsplit("_", 1)[1])
    probs = mg.batched_castings(n_inst)
    t_setup = time.perf_counter()
    b = fem.Batch(probs, args.precision, block_elems=args.block_elems, threads=args.threads)
    stream = torch.cuda.Stream()
    b.set_stream(stream.cuda_stream)
    dt = 0.9 * b.instance_stable_dt()
    b.advance(float(dt.min()))   # device set-up, graph of a one-step pattern
    t_setup = time.perf_counter() - t_setup
    tuned = autotune(b, args.autotune, args.autotune_steps, float(dt.min())) if args.autotune else None
    span = args.steps * float(dt.min())

    def counts(sp):
        return np.array([max(1, math.ceil(sp / d * (1.0 - 1e-12))) for d in dt])

    t_now = b.instance_times()[0].max()
    for _ in range(max(1, args.warmup // 3)):   # warm-up advances (graph capture)
        t_now += span
        b.advance(t_now)
    torch.cuda.synchronize()
    n = counts(span)
    tets = np.array([p.n_tets for p in probs], dtype=np.float64)
    updates = float((tets * n).sum())
    clocks = ClockSampler(0)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t_now += span
    ev0.record(stream)
    b.advance(t_now)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    post = 0
    while clocks.remaining() > 0.0:    # untimed advances so the clock record has samples
        t_now += span
        b.advance(t_now)
        torch.cuda.synchronize()
        post += 1
    clk = clocks.stop()
    if clk is not None:
        clk["untimed_advances_after"] = post
    value = updates / (ms / 1e3)
    info = b.info()
    # kernels in the timed advance: per step, two per run of consecutive
    # plan positions still stepping
    nk = n[b.plan("inst_order")]
    launches = 0
    for st in range(int(n.max())):
        act = nk > st
        launches += 2 * int(act[0] + np.count_nonzero(act[1:] & ~act[:-1]))

    # per-kernel device times of a step of every instance (each at the
    # smallest instance step, stable for all): events around each kernel
    kms = b.step_profile(args.profile_steps, float(dt.min())) / max(1, args.profile_steps)
    s = 4 if args.precision == "fp32" else 8
    peak, peak_kind = hbm_peak()
    E_all, N_all, n_int = int(tets.sum()), info["n_nodes"], info["n_interior_nodes"]
    alg = [E_all * (16 + 6 * s) + n_int * 4 * s, (N_all - n_int) * 4 * s]
    names = ["k_block_step", "k_shared_update"]
    k_dom = int(np.argmax(kms))
    achieved = alg[k_dom] / (kms[k_dom] / 1e3) / 1e9
    adv_alg = (16 + 6 * s + (N_all / E_all) * 4 * s) * value / 1e9
    roofline = {"bound": "hbm", "kernel": names[k_dom], "achieved": round(achieved, 1),
                "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": measured_traffic(names[k_dom], args.precision, "block",
                                            E_all if k_dom == 0 else N_all, scope="batch"),
                "peak_source": peak_kind, "alg_bytes_per_launch": int(alg[k_dom]),
                "kernel_ms": {nm: round(float(v), 4) for nm, v in zip(names, kms)},
                "launch": "all instances stepping",
                "advance": {"achieved": round(adv_alg, 1), "frac": round(adv_alg / peak, 4),
                            "note": "whole timed advance at 42.7 B per tet-update (FP32)"}}

    # end to end through the C ABI: every advance uploads the whole batch's
    # state from pinned host memory, advances every instance by the same
    # span and reads all temperatures back (pipelined calls, one sync)
    e2e = None
    if not args.no_e2e:
        ke = max(2, min(args.e2e_steps, 10))
        io_dt = torch.float32 if args.precision == "fp32" else torch.float64
        E64 = torch.empty(N_all, dtype=torch.float64)
        b.state(E64.numpy())
        E_io = E64.to(io_dt).pin_memory()
        T_io = [torch.empty(N_all, dtype=io_dt, pin_memory=True) for _ in range(2)]

        def loop(k, t):
            for i in range(k):
                b.set_state_async(E_io, 0, 0.0)
                t += span
                b.advance(t)
                b.temperature_async(T_io[i % 2])
            b.sync()
            return t

        t_now = loop(1, t_now)
        t0 = time.perf_counter()
        t_now = loop(ke, t_now)
        el = time.perf_counter() - t0
        isz = E_io.element_size()
        e2e = {"value": updates * ke / el, "unit": "tet-updates/s",
               "h2d_bytes_per_step": N_all * isz, "d2h_bytes_per_step": N_all * isz,
               "steps": ke, "step": "one fem_advance of every instance",
               "api": f"fem_set_state_async{'_f32' if isz == 4 else ''} + fem_advance + "
                      f"fem_get_temperature_async{'_f32' if isz == 4 else ''}, fem_sync at the end"}
    b.close()
    seq = None
    if not args.no_sequential:
        # the same instances one after another, each its own mesh and steps
        tot = 0.0
        for i, p in enumerate(probs):
            with fem.Mesh(p, args.precision, reorder=args.reorder, block_elems=args.block_elems,
                          threads=args.threads) as m:
                m.set_stream(stream.cuda_stream)
                c = int(n[i])
                m.step(1, span / c)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                m.step(c, span / c)
                e1.record(stream)
                torch.cuda.synchronize()
                tot += e0.elapsed_time(e1)
        seq = updates / (tot / 1e3)
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline_batch(probs, args.cpu_seconds)
    line = {
        "metric": "tet-element updates/s", "value": value, "unit": "tet-updates/s",
        "n_gpus": 1, "steps": int(n.max()), "warmup": args.warmup, "ms_per_step": ms / n.max(),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n_instances": n_inst,
                   "n_tets": int(tets.sum()), "n_nodes": info["n_nodes"],
                   "instance_tets_min": int(tets.min()), "instance_tets_max": int(tets.max()),
                   "steps_per_instance_min": int(n.min()), "steps_per_instance_max": int(n.max()),
                   "tet_updates": updates, "ms_advance": ms, "n_blocks": info["n_blocks"],
                   "threads": info["threads"], "precision": args.precision,
                   "sequential_value": seq, "autotune": tuned,
                   "l2": "inputs larger than L2 (no flush)", "setup_s": round(t_setup, 1)},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
        "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)


def run_surrogate(args):
    """The learned surrogate (16 explicit steps per network evaluation) with
    the plain solver as judge and fallback, against the plain FP32 solver,
    on unseen full-size castings: both solve from the pour until the casting
    has solidified (plus 10 %); value = plain time / surrogate time (CUDA
    events) over those solves, with the max nodal error and the
    solidification-time error beside it."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1005_3158_gb300 import fem
    from paper_1005_3158_gb300 import meshgen as mg
    from paper_1005_3158_gb300 import surrogate as sgd
    path = args.params or sgd.PARAMS_FILE
    if not os.path.exists(path):
        print(json.dumps({"metric": "surrogate speedup at <=2K max nodal error",
                          "unavailable": f"no trained parameters at {os.path.basename(path)}"}))
        return
    theta = np.load(path).astype(np.float32)
    geoms = mg.surrogate_eval_set(10)[:max(1, args.n_eval)]
    clocks = ClockSampler(0)
    clocks.start()
    res = [sgd.evaluate(p, theta, args.judge_every, (args.tol,), log=lambda *a: None) for p in geoms]
    clk = clocks.stop()
    ms_p = sum(r["ms_plain"] for r in res)
    ms_s = sum(r["ms_surrogate"] for r in res)
    value = ms_p / ms_s
    # per-kernel device times of the network on the first geometry
    p = geoms[0]
    m = fem.Mesh(p, "fp32", reorder=1)
    dt = 0.9 * m.stable_dt()
    sg = fem.Surrogate(m, dt)
    sg.set_params(theta)
    sg.profile(3)
    kms = sg.profile(args.profile_steps) / max(1, args.profile_steps)
    N, nnz = sg.n_nodes, sg.n_edges
    rows = (N + 127) // 128 * 128
    # fem_surrogate_profile's groups: kernel, launches per evaluation and
    # algorithmic bytes per launch (bf16 activations, FP32 graph data)
    groups = [
        # T(E) + features: E, C, Lc, phase byte and the Robin terms per node,
        # T and f read again through the CSR (column + weight per edge), x
        # written (16 bf16)
        ("k_sg_tf + k_sg_feat", 2, N * (4 + 4 + 4 + 1 + 8 + 8 + 8 + 32) + nnz * 8),
        # x read, h0 (64 bf16) and phi_1 (32 bf16) written
        ("k_sg_encode", 1, rows * (32 + 128 + 64)),
        # phi read once per node, m written (32 bf16 each), the CSR (int32
        # column + FP32 weight per edge, row pointer) and wsum, s per node
        ("k_sg_msg_tile", 3, N * (64 + 64 + 4 + 8) + nnz * 8),
        # [h; m] read, h and the next phi written
        ("k_sg_layer<false>", 2, rows * (128 + 64 + 128 + 64)),
        # [h; m], E and C read, E' written
        ("k_sg_layer<true>", 1, rows * (128 + 64) + N * (4 + 4 + 4)),
    ]
    per_launch = [kms[i] / groups[i][1] for i in range(5)]
    k_dom = int(np.argmax(kms))
    peak, peak_kind = hbm_peak()
    name, nl, alg = groups[k_dom]
    ach = alg / (per_launch[k_dom] / 1e3) / 1e9
    # the dense layers' contraction on tcgen05 (U_l [h; m] and P_{l+1} h)
    flops_layer = rows * 2 * (96 * 64 + 64 * 32)
    roofline = {"bound": "hbm", "kernel": name, "achieved": round(ach, 1),
                "peak": peak, "unit": "GB/s", "frac": round(ach / peak, 4), "traffic": None,
                "peak_source": peak_kind, "alg_bytes_per_launch": int(alg),
                "launches_per_evaluation": nl,
                "kernel_ms_per_launch": {g[0]: round(float(v), 4) for g, v in zip(groups, per_launch)},
                "k_sg_layer<false>": {
                    "alg_bytes_per_launch": int(groups[3][2]),
                    "frac_hbm": round(groups[3][2] / (per_launch[3] / 1e3) / 1e9 / peak, 4),
                    "flops_per_launch": int(flops_layer),
                    "achieved_tflops": round(flops_layer / (per_launch[3] / 1e3) / 1e12, 2),
                    "note": "dense per-node layers on tcgen05 (BF16, FP32 accumulation in TMEM); "
                            "the message sums gather on CUDA cores"}}
    # end to end through the C ABI with host buffers: upload the pour state
    # (FP32, pinned), solve, read the temperatures back; plain vs surrogate
    e2e = None
    if not args.no_e2e:
        E64 = torch.empty(N, dtype=torch.float64)
        m.set_temperature(p.T0)
        m.state(E64.numpy())
        E_h = E64.to(torch.float32).pin_memory()
        T_h = torch.empty(N, dtype=torch.float32, pin_memory=True)
        n_macro = res[0]["macro_steps"]
        times = {}
        for name in ("plain", "surrogate"):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            m.set_state_async(E_h, 0, 0.0)
            if name == "plain":
                m.step(16 * n_macro, dt)
            else:
                sg.solve(n_macro, args.judge_every, args.tol)
            m.temperature_async(T_h)
            m.sync()
            times[name] = time.perf_counter() - t0
        e2e = {"value": times["plain"] / times["surrogate"], "unit": "x",
               "h2d_bytes_per_step": N * 4, "d2h_bytes_per_step": N * 4,
               "step": f"one whole solve ({n_macro} macro steps) of {p.name}",
               "seconds_plain": times["plain"], "seconds_surrogate": times["surrogate"]}
    sg.close()
    m.close()
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline_surrogate(theta)
    line = {
        "metric": "surrogate speedup at <=2K max nodal error (hybrid surrogate vs plain FP32 "
                  "solver, same GPU, same simulated time)",
        "value": value, "unit": "x", "n_gpus": 1, "steps": sum(r["steps"] for r in res),
        "warmup": 2, "ms_per_step": ms_s / sum(r["steps"] for r in res),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": "surrogate_flanged", "geometries": [r["geometry"] for r in res],
                   "n_tets": res[0]["n_tets"], "n_nodes": res[0]["n_nodes"],
                   "judge_every": args.judge_every, "tol_K": args.tol,
                   "params": os.path.basename(path),
                   "max_err_K": max(r["max_err_K"] for r in res),
                   "solid_time_rel_err": max((r["solid_time_rel_err"] or 0.0) for r in res),
                   "macro_by_surrogate": sum(r["macro_by_surrogate"] for r in res),
                   "macro_by_solver": sum(r["macro_by_solver"] for r in res),
                   "ms_per_16_steps_plain": ms_p / sum(r["macro_steps"] for r in res),
                   "ms_per_16_steps_surrogate": ms_s / sum(r["macro_steps"] for r in res),
                   "ms_per_16_steps_network": float(np.mean([r["ms_per_16_steps_network"] for r in res])),
                   "per_geometry": [{k: v for k, v in r.items() if k not in ("err_K_by_macro", "by_tol")}
                                    for r in res],
                   "l2": "inputs larger than L2 (no flush)"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
        "gpu_launches": None,
    }
    print(json.dumps(line), flush=True)


def cpu_baseline_surrogate(theta, seconds: float = 10.0):
    """The surrogate oracle (numpy forward pass, bf16 emulation) on a small
    casting of the same family, timed on the host: tet-updates/s it
    advances (16 steps per pass)."""
    import numpy as np
    from oracle import surrogate as osg
    from paper_1005_3158_gb300 import meshgen as mg
    p = mg.flanged_variant(4000, 0.2)
    o = __import__("oracle").OracleProblem(p)
    dt = 0.9 * o.stable_dt()
    g = osg.SurrogateGraph(p, dt)
    o.set_temperature(p.T0)
    E = o.enthalpy()
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds or n == 0:
        E, _ = osg.forward(theta, g, E, emulate=True)
        n += 1
    el = time.perf_counter() - t0
    return {"value": p.n_tets * 16 * n / el, "unit": "tet-updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{p.name} ({p.n_tets} tets), {n} surrogate forward passes of the numpy "
                      f"oracle (16 steps each), {el:.1f} s"}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload.startswith("batched_castings_"):
        run_batched(args)
        return
    if args.workload == "surrogate_flanged":
        run_surrogate(args)
        return
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_1005_3158_gb300 import fem

    p = make_problem(args.workload)
    if args.physics == "kt":
        # k(T) of the alloy (material 0) and the steel (1): piecewise linear
        # between the table points, constant beyond them
        p.k_tables = ((0, [300.0, 600.0, 821.0, 913.0], [150.0, 160.0, 140.0, 90.0]),
                      (1, [300.0, 900.0], [30.0, 26.0]))
    t_setup = time.perf_counter()
    mesh = fem.Mesh(p, args.precision, reorder=args.reorder, variant=args.variant,
                    block_elems=args.block_elems, threads=args.threads,
                    formulation="apparent" if args.physics == "apparent" else "enthalpy")
    dt = 0.9 * mesh.stable_dt()
    stream = torch.cuda.Stream()
    mesh.set_stream(stream.cuda_stream)
    mesh.step(1, dt)
    t_setup = time.perf_counter() - t_setup
    tuned = autotune(mesh, args.autotune, args.autotune_steps, dt) if args.autotune else None
    info = mesh.info()
    E, N = p.n_tets, p.n_nodes

    # warm-up, then K timed steps between barriers, CUDA events on the stream
    clocks = ClockSampler(local)
    clocks.start()
    mesh.step(args.warmup, dt)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    mesh.step(args.steps, dt)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    post = 0
    while clocks.remaining() > 0.0:    # untimed steps so the clock record has samples
        mesh.step(32, dt)
        torch.cuda.synchronize()
        post += 32
    clk = clocks.stop()
    if clk is not None:
        clk["untimed_steps_after"] = post
    ms = max_over_ranks(ms, world, "cuda")
    value = job_throughput(E, args.steps, world, ms / 1e3)
    kernels_per_step = 2 if info["n_shared_nodes"] > 0 or args.variant != "block" else 1
    if args.variant != "block":
        kernels_per_step = 3
    n_launch_per_step = kernels_per_step
    if args.variant == "colored":
        n_launch_per_step = 2 + info["n_colors"]

    # per-kernel device times (separate pass with events around each kernel)
    kms = mesh.step_profile(args.profile_steps, dt) / max(1, args.profile_steps)
    s = 4 if args.precision == "fp32" else 8
    peak, peak_kind = hbm_peak()
    if args.variant == "block":
        n_int = info["n_interior_nodes"]
        # algorithmic bytes: int32 connectivity + six stored conductances per
        # tet, E read+write and C, Lc per node (stored-K^e EBE)
        alg = [E * (16 + 6 * s) + n_int * 4 * s, (N - n_int) * 4 * s]
        names = ["k_block_step", "k_shared_update"]
    else:
        alg = [N * 2 * s + N * 4 * s, E * (16 + 6 * s), N * 4 * s]
        names = ["k_flat_temperature", "k_flat_elements", "k_flat_update"]
    k_dom = int(np.argmax(kms))
    achieved = alg[k_dom] / (kms[k_dom] / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": names[k_dom], "achieved": round(achieved, 1),
                "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": measured_traffic(names[k_dom], args.precision, args.variant,
                                            E if names[k_dom] != "k_shared_update" else N),
                "peak_source": peak_kind,
                "alg_bytes_per_launch": int(alg[k_dom]),
                "kernel_ms": {n: round(float(v), 4) for n, v in zip(names, kms)},
                "step_alg_bytes_per_tet": round((E * (16 + 6 * s) + N * 4 * s) / E, 2)}

    if args.precision == "fp64" and args.variant == "block":
        # FP64 on GB300 is bound by its FP64 pipe (2 FMA per clock per SM),
        # not by HBM: report the block kernel against that pipe's peak.
        # Algorithmic FP64 flops: 28 per tet (pass 2: 6 differences, 6
        # products, 12 corner-sum adds; pass 3: 4 slot adds), 5 per interior
        # node (T(E), update), 3 per shared-node copy (T(E)).
        flops = E * 28 + info["n_interior_nodes"] * 5 + info["n_shared_copies"] * 3
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        mhz = (clk or {}).get("sm_max_mhz") or 2070.0
        fpeak = sms * 2 * 2 * mhz * 1e6 / 1e9
        fach = flops / (kms[0] / 1e3) / 1e9
        roofline = {"bound": "alu", "kernel": "k_block_step", "achieved": round(fach, 1),
                    "peak": round(fpeak, 1), "unit": "GFLOP/s", "frac": round(fach / fpeak, 4),
                    "traffic": roofline["traffic"],
                    "peak_source": f"derived: {sms} SMs x 2 FP64 FMA/clock x {mhz:.0f} MHz",
                    "alg_flops_per_launch": int(flops), "hbm": {
                        "achieved": roofline["achieved"], "peak": peak, "unit": "GB/s",
                        "frac": roofline["frac"]},
                    "kernel_ms": roofline["kernel_ms"]}

    # end to end through the C ABI with pinned host buffers: every step
    # uploads the state, steps once and reads the temperatures back.  The
    # headline uses the pipelined calls (each step's copies overlap the
    # neighbouring steps) with host arrays in the mesh's own precision;
    # the pipelined loop with FP64 arrays and the serial loop through the
    # synchronous (FP64) calls are reported beside it.
    e2e = None
    if not args.no_e2e:
        ke = args.e2e_steps or args.steps
        io_dt = torch.float32 if args.precision == "fp32" else torch.float64
        E64 = torch.empty(N, dtype=torch.float64, pin_memory=True)
        mesh.state(E64.numpy())
        E_io = E64.to(io_dt).pin_memory()
        T64 = [torch.empty(N, dtype=torch.float64, pin_memory=True) for _ in range(2)]
        T_io = [torch.empty(N, dtype=io_dt, pin_memory=True) for _ in range(2)]

        def serial(n):
            for _ in range(n):
                mesh.set_state(E64, 0, 0.0)
                mesh.step(1, dt)
                mesh.temperature(T64[0])

        def pipelined(E_h, T_h):
            def run(n):
                for k in range(n):
                    mesh.set_state_async(E_h, 0, 0.0)
                    mesh.step(1, dt)
                    mesh.temperature_async(T_h[k % 2])
                mesh.sync()
            return run

        rates = {}
        for name, loop in (("serial", serial), ("pipelined_f64", pipelined(E64, T64)),
                           ("pipelined", pipelined(E_io, T_io))):
            loop(3)
            if world > 1:
                dist.barrier()
            t0 = time.perf_counter()
            loop(ke)
            el = max_over_ranks(time.perf_counter() - t0, world, "cuda")
            rates[name] = job_throughput(E, ke, world, el)
        isz = E_io.element_size()
        e2e = {"value": rates["pipelined"], "unit": "tet-updates/s",
               "h2d_bytes_per_step": N * isz, "d2h_bytes_per_step": N * isz, "steps": ke,
               "api": f"fem_set_state_async{'_f32' if isz == 4 else ''} + fem_step + "
                      f"fem_get_temperature_async{'_f32' if isz == 4 else ''}, fem_sync at the end",
               "pipelined_f64_value": rates["pipelined_f64"], "serial_value": rates["serial"]}

    cpu = thr = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        cpu, sp, sname, sdt = cpu_baseline(args.workload, args.cpu_seconds)
        if not args.no_cpu_threaded:
            try:
                thr = cpu_threaded(sp, sname, sdt, args.cpu_threaded_seconds)
            except Exception as e:   # noqa: BLE001  (no OpenMP compiler on the host)
                thr = {"unavailable": f"{type(e).__name__}: {e}"[:200]}

    if rank == 0:
        line = {
            "metric": "tet-element updates/s", "value": value, "unit": "tet-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "n_tets": E, "n_nodes": N,
                       "n_faces": p.n_faces, "variant": args.variant, "physics": args.physics,
                       "precision": args.precision, "reorder": args.reorder,
                       "n_blocks": info["n_blocks"], "threads": info["threads"],
                       "ctas_per_sm": info["ctas_per_sm"], "smem_per_cta": info["smem_per_cta"],
                       "block_elems": args.block_elems,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (no flush)",
                       "dt_s": dt, "setup_s": round(t_setup, 1), "autotune": tuned},
            "roofline": roofline, "cpu_baseline": cpu, "cpu_threaded": thr, "e2e": e2e,
            "clocks": clk, "gpu_launches": n_launch_per_step * args.steps,
        }
        print(json.dumps(line), flush=True)
    mesh.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
