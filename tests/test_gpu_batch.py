"""GPU batches: every instance of a batch against its own FP64 oracle run.

fem_advance(t_end) gives instance i n_i = ceil((t_end - t_i) / dt_i) equal
steps of (t_end - t_i) / n_i; the oracle takes the same steps.  Tolerances
as for single meshes (FP64 1e-9 K, FP32 0.05 K).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1005_3158_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 0.05}


@pytest.fixture(scope="module")
def fem():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1005_3158_gb300 import fem as f
    return f


def _steps(span, dt):
    if not span > 0:
        return 0, 0.0
    c = max(1, math.ceil(span / dt * (1.0 - 1e-12)))
    return c, span / c


def _parts():
    return [mg.random_small(s, nx=nx, ny=ny, nz=nz, n_mat=3)
            for s, (nx, ny, nz) in zip([21, 22, 23, 24, 25],
                                       [(5, 4, 4), (7, 6, 5), (3, 3, 4), (8, 5, 5), (6, 6, 3)])]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_advance_matches_oracle(fem, prec):
    probs = _parts()
    oracles = []
    for p in probs:
        o = oracle.OracleProblem(p)
        o.set_temperature(p.T0)
        oracles.append(o)
    with fem.Batch(probs, prec, block_elems=96) as b:
        dt = 0.9 * b.instance_stable_dt()
        t_end = 25.0 * float(np.median(dt))
        t_prev = np.zeros(len(probs))
        for rnd in range(3):   # the second and third advance reuse the graph
            t_goal = t_end * (rnd + 1)
            b.advance(t_goal)
            T = b.temperature()
            t, n = b.instance_times()
            for i, (p, o) in enumerate(zip(probs, oracles)):
                c, dtp = _steps(t_goal - t_prev[i], dt[i])
                o.step(c, dtp)
                assert t[i] == t_goal
                err = np.abs(b.instance_temperature(i, T) - o.temperature()).max()
                assert err <= TOL[prec], f"advance {rnd} instance {i}: {err:.3e} K"
            t_prev[:] = t_goal
        for i, o in enumerate(oracles):
            U, U0, Qb, lat = b.instance_energy(i)
            eo = o.energy()
            rel = 1e-12 if prec == "fp64" else 1e-5
            assert abs(U - U0 - Qb) <= rel * abs(U0)
            assert U == pytest.approx(eo[0], rel=1e-12 if prec == "fp64" else 1e-6)
            assert Qb == pytest.approx(eo[2], rel=1e-9 if prec == "fp64" else 1e-3, abs=1e-6 * abs(U0))


def test_advance_unordered_steps(fem):
    """Per-instance steps that do not follow the plan order: every step
    launches once per run of instances still stepping."""
    probs = _parts()
    with fem.Batch(probs, "fp64", block_elems=64) as b:
        stable = b.instance_stable_dt()
        rng = np.random.default_rng(4)
        dt = stable * rng.uniform(0.2, 0.9, size=len(probs))
        b.set_instance_dt(dt)
        t_end = 12.0 * float(stable.max())
        b.advance(t_end)
        T = b.temperature()
        _, n = b.instance_times()
        for i, p in enumerate(probs):
            o = oracle.OracleProblem(p)
            o.set_temperature(p.T0)
            c, dtp = _steps(t_end, dt[i])
            assert n[i] == c
            o.step(c, dtp)
            assert np.abs(b.instance_temperature(i, T) - o.temperature()).max() <= 1e-9


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_step_is_bitwise_the_parts(fem, prec):
    """Every instance is planned exactly as it would be alone, so fem_step on
    the batch reproduces each part's own run bit for bit."""
    probs = _parts()
    with fem.Batch(probs, prec, block_elems=80) as b:
        dt = 0.9 * float(b.instance_stable_dt().min())
        b.step(40, dt)
        T = b.temperature()
        for i, p in enumerate(probs):
            with fem.Mesh(p, prec, block_elems=80) as m:
                m.step(40, dt)
                assert np.array_equal(b.instance_temperature(i, T), m.temperature())


def test_batched_castings_fp32(fem):
    probs = mg.batched_castings(6, seed=11, lo=2e4, hi=6e4)
    with fem.Batch(probs, "fp32") as b:
        dt = 0.9 * b.instance_stable_dt()
        t_end = 20.0 * float(dt.min())
        b.advance(t_end)
        T = b.temperature()
        for i, p in enumerate(probs):
            o = oracle.OracleProblem(p)
            o.set_temperature(p.T0)
            c, dtp = _steps(t_end, dt[i])
            o.step(c, dtp)
            err = np.abs(b.instance_temperature(i, T) - o.temperature()).max()
            assert err <= TOL["fp32"], f"instance {i}: {err:.3e} K"
