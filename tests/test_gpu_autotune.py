"""fem_autotune on the GPU: it picks one of the candidates, keeps the state,
time, step count and energy accounts it found, and later steps still match
the FP64 oracle."""
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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_autotune_keeps_state_and_parity(fem, prec):
    p = mg.random_small(41, nx=9, ny=8, nz=7, n_mat=3)
    o = oracle.OracleProblem(p)
    o.set_temperature(p.T0)
    dt = 0.9 * o.stable_dt()
    with fem.Mesh(p, prec, block_elems=2048) as m:
        m.step(30, dt)
        T0 = m.temperature()
        E0, s0, t0 = m.state()
        U0 = m.energy()
        cands = [96, 192, 384, 768]
        best, ms = m.autotune(cands, steps=5, dt=dt)
        assert 0 <= best < len(cands)
        assert np.isfinite(ms).all() and (ms > 0).all() and ms[best] == ms.min()
        assert m.info()["max_block_elems"] <= cands[best]
        E1, s1, t1 = m.state()
        assert np.array_equal(E0, E1) and s1 == s0 and t1 == t0
        assert np.array_equal(T0, m.temperature())
        U1 = m.energy()
        assert U1[1] == U0[1] and U1[2] == U0[2]
        assert U1[0] == pytest.approx(U0[0], rel=1e-12)
        m.step(50, dt)
        o.step(80, dt)
        err = np.abs(m.temperature() - o.temperature()).max()
        assert err <= TOL[prec], f"{err:.3e} K"
        U = m.energy()
        assert abs(U[0] - U[1] - U[2]) <= (1e-12 if prec == "fp64" else 1e-5) * abs(U[1])


def test_autotune_skips_candidates_that_do_not_fit(fem):
    p = mg.unit_cube(12)
    with fem.Mesh(p, "fp64") as m:
        dt = 0.9 * m.stable_dt()
        best, ms = m.autotune([12288, 512], [0, 256], steps=3, dt=dt)
        assert best == 1 and math.isinf(ms[0]) and np.isfinite(ms[1])
        assert m.info()["threads"] == 256
        with pytest.raises(fem.FemError) as e:
            m.autotune([12288], steps=3, dt=dt)
        assert e.value.status == fem.FEM_EINVAL
        m.step(5, dt)   # the mesh still steps with the partition it kept


def test_autotune_batch(fem):
    probs = [mg.random_small(s, nx=nx, ny=ny, nz=nz, n_mat=2)
             for s, (nx, ny, nz) in zip([42, 43, 44], [(6, 5, 4), (4, 4, 4), (7, 5, 5)])]
    with fem.Batch(probs, "fp64", block_elems=512) as b:
        dt = 0.9 * b.instance_stable_dt()
        t1 = 10.0 * float(dt.min())
        b.advance(t1)
        times0, n0 = b.instance_times()
        e0 = [b.instance_energy(i) for i in range(len(probs))]
        best, ms = b.autotune([64, 128, 256], steps=4, dt=float(dt.min()))
        times1, n1 = b.instance_times()
        assert np.array_equal(times0, times1) and np.array_equal(n0, n1)
        for i in range(len(probs)):
            e1 = b.instance_energy(i)
            assert e1[1] == e0[i][1] and e1[2] == pytest.approx(e0[i][2], rel=1e-13, abs=1e-9)
            assert e1[0] == pytest.approx(e0[i][0], rel=1e-12)
        t2 = 2.0 * t1
        b.advance(t2)
        T = b.temperature()
        for i, p in enumerate(probs):
            o = oracle.OracleProblem(p)
            o.set_temperature(p.T0)
            for span in (t1, t2 - t1):
                c = max(1, math.ceil(span / dt[i] * (1.0 - 1e-12)))
                o.step(c, span / c)
            assert np.abs(b.instance_temperature(i, T) - o.temperature()).max() <= 1e-9
