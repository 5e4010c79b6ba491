"""Training and evaluation driver of the learned surrogate (fem_surrogate_*).

Every computation runs in libfem's kernels: the explicit solver generates
the training trajectories, the surrogate's own CUDA kernels train and
evaluate the network.  PyTorch only holds device memory (the snapshot
pairs) and picks which pair each training step uses.

    python -m paper_1005_3158_gb300.surrogate train --out params.npy
    python -m paper_1005_3158_gb300.surrogate eval --params params.npy

Training data: ``meshgen.surrogate_training_set`` castings (the flanged
family at the casting workload's hex spacing) advanced together as one
batch from the pour, every instance at the same step (0.9 of the smallest
stable step); a pair (E_n, E_{n+16}) is recorded every ``every`` steps until
the castings have solidified.  Evaluation: ``meshgen.surrogate_eval_set``
full-size castings, each run twice from the pour, once by the plain FP32
solver and once by the surrogate with the solver as judge and fallback;
max nodal temperature difference and the casting's solidification time
(the last alloy node to fall below the solidus, linearly interpolated
between macro steps) are compared, and both runs are timed with CUDA
events.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

from . import fem
from . import meshgen as mg

PARAMS_FILE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "surrogate_params.npy")
MACRO = 16
MAX_BACKOFF = 6   # fem_surrogate_solve: largest doubling of the span after failed judgements


def param_shapes():
    """(name, shape) of the flat parameter vector, in the order fem.h gives."""
    shapes = [("W_in", (64, 16)), ("b_in", (64,))]
    for l in range(1, 4):
        shapes += [(f"P{l}", (32, 64)), (f"p{l}", (32,)), (f"U{l}", (64, 96)), (f"u{l}", (64,))]
    shapes += [("D1", (64, 64)), ("d1", (64,)), ("d2", (64,)), ("d2b", (1,))]
    assert sum(int(np.prod(s)) for _, s in shapes) == fem.FEM_SG_N_PARAMS
    return shapes


def _sync():
    import torch
    torch.cuda.synchronize()


def generate_pairs(probs, every=16, max_steps=4800, log=print):
    """Advance the castings as one batch from the pour and record (E_n,
    E_{n+16}) pairs on the device every `every` steps until the latent heat
    left is below 1e-4 of the initial one in every instance, after at least
    2400 steps (or max_steps).  Returns (batch, surrogate, pairs, dt)."""
    import torch
    b = fem.Batch(probs, "fp32")
    dt = 0.9 * float(b.instance_stable_dt().min())
    b.set_instance_dt(np.full(len(probs), dt))
    s = fem.Surrogate(b)
    lat0 = np.array([b.instance_energy(i)[3] for i in range(len(probs))])
    pairs = []
    steps = 0
    t0 = time.time()
    while steps < max_steps:
        Ea = torch.empty(s.n_nodes, dtype=torch.float32, device="cuda")
        Eb = torch.empty_like(Ea)
        s.read_state(Ea)
        b.step(MACRO, dt)
        s.read_state(Eb)
        pairs.append((Ea, Eb))
        b.step(every - MACRO, dt)
        steps += every
        if len(pairs) % 25 == 0:
            lat = np.array([b.instance_energy(i)[3] for i in range(len(probs))])
            frac = float((lat / np.maximum(lat0, 1e-30)).max())
            log(f"  {steps} steps, {len(pairs)} pairs, latent left <= {frac:.4f}, "
                f"{time.time() - t0:.1f} s")
            if frac < 1e-4 and steps >= 2400:
                break
    _sync()
    return b, s, pairs, dt


def train(s, pairs, iters=3000, lr0=1e-3, lr1=1e-5, seed=5, init=None, skip_first=0,
          per_step=1, push=0.0, log=print):
    """Adam on random pairs (each a whole batch snapshot), per_step pairs
    accumulated per step, cosine learning-rate decay from lr0 to lr1; the
    first skip_first pairs (the steep transient right after the pour, which
    the hybrid solve leaves to the explicit solver) are not used.  With
    probability `push` a sample is a pushforward pair instead: the network's
    own prediction from pair k's input, trained towards the solver's state
    one macro step later (pair k + 1's target), so that the network learns
    to correct the errors its own steps make (the pairs are consecutive
    macro steps).  Returns the loss history."""
    import torch
    theta = mg.surrogate_init(param_shapes(), seed=seed) if init is None else init
    s.set_params(theta)
    rng = np.random.default_rng(seed)
    pairs = pairs[skip_first:]
    scratch = torch.empty_like(pairs[0][0])
    hist = []
    t0 = time.time()
    for it in range(iters):
        lr = lr1 + 0.5 * (lr0 - lr1) * (1.0 + math.cos(math.pi * it / max(1, iters - 1)))
        want = it % 50 == 0 or it == iters - 1
        losses = []
        for q in range(per_step):
            if push > 0.0 and rng.random() < push and len(pairs) > 1:
                k = int(rng.integers(len(pairs) - 1))
                s.predict(pairs[k][0], scratch)
                losses.append(s.accumulate(scratch, pairs[k + 1][1], want_loss=want))
            else:
                Ea, Eb = pairs[int(rng.integers(len(pairs)))]
                losses.append(s.accumulate(Ea, Eb, want_loss=want))
        s.apply(lr)
        if want:
            loss = float(np.mean(losses))
            hist.append((it, loss))
            if it % 500 == 0 or it == iters - 1:
                log(f"  iter {it}: loss {loss:.4g}, lr {lr:.2e}, {time.time() - t0:.1f} s")
    _sync()
    return hist


def _solid_times(T_hist, times, alloy, Ts):
    """Per alloy node the first time its temperature reaches Ts or below,
    linearly interpolated between the recorded times (inf if never)."""
    T = np.asarray(T_hist)[:, alloy]
    out = np.full(T.shape[1], np.inf)
    for k in range(1, T.shape[0]):
        hit = (T[k] <= Ts) & (T[k - 1] > Ts) & ~np.isfinite(out)
        if hit.any():
            a, b = T[k - 1, hit], T[k, hit]
            out[hit] = times[k - 1] + (times[k] - times[k - 1]) * (a - Ts) / (a - b)
    out[(T[0] <= Ts)] = times[0]
    return out


def _timed(fn):
    import torch
    stream = torch.cuda.current_stream()
    _sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    _sync()
    return e0.elapsed_time(e1)


class HybridPolicy:
    """The macro-step policy of fem_surrogate_solve, step by step: macro
    step 0 is judged (if judge_every > 0); after a passed judgement the
    network takes the next judge_every - 1 macro steps, after a failed one
    the solver does, the span doubling with each further consecutive
    failure (up to 2^MAX_BACKOFF judge_every); the step after the span is
    judged again.  action(k) -> "judge" | "solver" | "network"; report
    every judged step's outcome with judged(k, passed)."""

    def __init__(self, judge_every):
        self.J = int(judge_every)
        self.next_judge = 0
        self.plain_until = 0
        self.fails = 0

    def action(self, k):
        if self.J > 0 and k == self.next_judge:
            return "judge"
        return "solver" if k < self.plain_until else "network"

    def judged(self, k, passed):
        span = self.J
        if passed:
            self.fails = 0
        else:
            span = self.J << min(self.fails, MAX_BACKOFF)
            self.fails += 1
            self.plain_until = k + span
        self.next_judge = k + span


def evaluate(p, theta, judge_every=8, tols=(2.0,), max_macro=4000, log=print):
    """One geometry: plain FP32 solve from the pour until the casting has
    solidified (plus 10 %); then, for every tolerance, the surrogate's
    hybrid solve over the same macro steps read back every macro step (max
    nodal difference, solidification time) and timed again without
    read-backs; the plain solve and the network alone are timed too.  The
    result's top-level figures are those of the first tolerance; all are in
    res["by_tol"]."""
    Ts = float(p.materials[0][4])
    alloy = np.zeros(p.n_nodes, bool)
    alloy[p.tets[p.mat == 0].ravel()] = True
    res = {"geometry": p.name, "n_tets": p.n_tets, "n_nodes": p.n_nodes}
    m = fem.Mesh(p, "fp32", reorder=1)
    dt = 0.9 * m.stable_dt()
    T_plain = [m.temperature().astype(np.float32)]
    k = 0
    while k < max_macro:
        m.step(MACRO, dt)
        k += 1
        T_plain.append(m.temperature().astype(np.float32))
        if T_plain[-1][alloy].max() <= Ts:
            break
    n_macro = min(max_macro, int(math.ceil(1.1 * k)))
    while k < n_macro:
        m.step(MACRO, dt)
        k += 1
        T_plain.append(m.temperature().astype(np.float32))
    m.close()
    times = np.arange(n_macro + 1) * MACRO * dt
    st_plain = _solid_times(T_plain, times, alloy, Ts)
    ts_p = float(st_plain.max())
    res.update({"dt": dt, "macro_steps": n_macro, "steps": n_macro * MACRO,
                "simulated_s": float(times[-1]), "solid_time_plain_s": ts_p})
    # timings: plain solver, network alone
    mm = fem.Mesh(p, "fp32", reorder=1)
    mm.step(2 * MACRO, dt)
    mm.set_temperature(p.T0)
    res["ms_plain"] = _timed(lambda: mm.step(n_macro * MACRO, dt))
    ss = fem.Surrogate(mm, dt)
    ss.set_params(theta)
    mm.set_temperature(p.T0)
    ss.advance(2)
    mm.set_temperature(p.T0)
    res["ms_per_16_steps_network"] = _timed(lambda: ss.advance(n_macro)) / n_macro
    res["ms_per_16_steps_plain"] = res["ms_plain"] / n_macro
    by_tol = {}
    for tol in tols:
        r = {"tol_K": tol}
        m2 = fem.Mesh(p, "fp32", reorder=1)
        s = fem.Surrogate(m2, dt)
        s.set_params(theta)
        T_sg = [m2.temperature().astype(np.float32)]
        err_t = [0.0]
        n_sg = n_pl = n_fail = 0
        worst_judge = 0.0
        # the policy of fem_surrogate_solve, one macro step at a time so that
        # every macro step can be read back
        pol = HybridPolicy(judge_every)
        for k in range(n_macro):
            act = pol.action(k)
            if act == "judge":
                _, b_, c, e = s.solve(1, 1, tol)
                n_pl += b_
                n_fail += c
                worst_judge = max(worst_judge, e)
                pol.judged(k, passed=not c)
            elif act == "solver":
                m2.step(MACRO, dt)
                n_pl += 1
            else:
                s.advance(1)
                n_sg += 1
            T_sg.append(m2.temperature().astype(np.float32))
            err_t.append(float(np.abs(T_sg[-1] - T_plain[k + 1]).max()))
        s.close()
        m2.close()
        ts_s = float(_solid_times(T_sg, times, alloy, Ts).max())
        r.update({"max_err_K": float(max(err_t)), "err_K_by_macro": err_t[::max(1, n_macro // 20)],
                  "solid_time_surrogate_s": ts_s,
                  "solid_time_rel_err": abs(ts_s - ts_p) / ts_p if math.isfinite(ts_p) else None,
                  "macro_by_surrogate": n_sg, "macro_by_solver": n_pl, "judge_failures": n_fail,
                  "max_judged_K": worst_judge})
        mm.set_temperature(p.T0)
        ss.solve(2, judge_every, tol)       # warm-up
        mm.set_temperature(p.T0)
        r["ms_surrogate"] = _timed(lambda: ss.solve(n_macro, judge_every, tol))
        r["ms_per_16_steps_surrogate"] = r["ms_surrogate"] / n_macro
        r["speedup"] = res["ms_plain"] / r["ms_surrogate"]
        by_tol[str(tol)] = r
        log(json.dumps({"geometry": p.name, **{k: v for k, v in r.items() if k != "err_K_by_macro"}}))
    ss.close()
    mm.close()
    res.update({k: v for k, v in by_tol[str(tols[0])].items()})
    res["by_tol"] = by_tol
    log(json.dumps({k: v for k, v in res.items() if k not in ("err_K_by_macro", "by_tol")}))
    return res


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train", "eval", "run"],
                    help="train, eval, or run: a plain surrogate advance of --macro macro "
                         "steps on one casting of --scale (for profilers)")
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--macro", type=int, default=4)
    ap.add_argument("--out", default=PARAMS_FILE)
    ap.add_argument("--params", default=PARAMS_FILE)
    ap.add_argument("--n-train", type=int, default=200)
    ap.add_argument("--every", type=int, default=16)
    ap.add_argument("--iters", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--skip-first", type=int, default=0)
    ap.add_argument("--per-step", type=int, default=1, help="pairs accumulated per Adam step")
    ap.add_argument("--push", type=float, default=0.0, help="fraction of pushforward pairs")
    ap.add_argument("--init", default="", help="start from these parameters")
    ap.add_argument("--n-eval", type=int, default=10)
    ap.add_argument("--judge-every", type=int, default=8)
    ap.add_argument("--tol", type=float, nargs="+", default=[2.0])
    ap.add_argument("--json", default="")
    a = ap.parse_args(argv)
    if a.cmd == "train":
        t0 = time.time()
        probs = mg.surrogate_training_set(a.n_train)
        print(f"training set: {len(probs)} castings, {sum(p.n_tets for p in probs)} tets", flush=True)
        b, s, pairs, dt = generate_pairs(probs, every=a.every)
        print(f"pairs: {len(pairs)} (dt {dt:.4g} s), {time.time() - t0:.1f} s", flush=True)
        init = np.load(a.init).astype(np.float32) if a.init else None
        hist = train(s, pairs, iters=a.iters, lr0=a.lr, init=init, skip_first=a.skip_first,
                     per_step=a.per_step, push=a.push)
        np.save(a.out, s.params())
        if a.json:
            with open(a.json, "w") as f:
                json.dump({"loss": hist, "pairs": len(pairs), "dt": dt,
                           "n_train": len(probs), "seconds": time.time() - t0}, f)
        s.close()
        b.close()
    elif a.cmd == "run":
        theta = np.load(a.params).astype(np.float32)
        p = mg.flanged_variant(4000, a.scale)
        m = fem.Mesh(p, "fp32", reorder=1)
        s = fem.Surrogate(m, 0.9 * m.stable_dt())
        s.set_params(theta)
        s.advance(a.macro)
        _sync()
        print(f"{p.name}: {p.n_tets} tets, {a.macro} surrogate macro steps")
        s.close()
        m.close()
    else:
        theta = np.load(a.params).astype(np.float32)
        out = [evaluate(p, theta, a.judge_every, tuple(a.tol)) for p in mg.surrogate_eval_set(a.n_eval)]
        if a.json:
            with open(a.json, "w") as f:
                json.dump(out, f)


if __name__ == "__main__":
    main(sys.argv[1:])
