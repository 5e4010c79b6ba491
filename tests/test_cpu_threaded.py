"""The threaded CPU baseline (OpenMP, colour-parallel element loop) that
bench.py times beside the GPU: it must compute the oracle's step (FP64 to
1e-9 K, FP32 to 0.05 K) and give the same bits for any thread count (each
colour's elements share no node, and every sum runs in a fixed order)."""
import numpy as np
import pytest

import oracle
from paper_1005_3158_gb300 import meshgen as mg

ct = pytest.importorskip("cpu_threaded")

TOL = {"fp64": 1e-9, "fp32": 0.05}


@pytest.mark.parametrize("seed", [31, 32])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_matches_oracle(seed, prec):
    p = mg.random_small(seed, nx=6, ny=5, nz=4, n_mat=3)
    o = oracle.OracleProblem(p)
    o.set_temperature(p.T0)
    dt = 0.9 * o.stable_dt()
    o.step(150, dt)
    with ct.ThreadedBaseline(p, prec, threads=2) as b:
        b.step(150, dt)
        err = np.abs(b.temperature() - o.temperature()).max()
    assert err <= TOL[prec], f"{prec}: {err:.3e} K"


def test_unit_cube_energy_and_colours():
    p = mg.unit_cube(10)
    o = oracle.OracleProblem(p)
    o.set_temperature(p.T0)
    dt = 0.9 * o.stable_dt()
    o.step(100, dt)
    with ct.ThreadedBaseline(p, "fp64", threads=3) as b:
        b.step(100, dt)
        assert b.energy() == pytest.approx(o.energy()[0], rel=1e-12)
        inf = b.info()
    # greedy colouring needs at most one colour more than the number of
    # elements that share a node with any one element; Kuhn meshes need ~30
    assert 1 < inf["colours"] <= 64 and inf["threads"] == 3


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_thread_count_invariance(prec):
    p = mg.random_small(33, nx=7, ny=6, nz=5, n_mat=2)
    o = oracle.OracleProblem(p)
    dt = 0.9 * o.stable_dt()
    out = []
    for th in (1, 2, 5):
        with ct.ThreadedBaseline(p, prec, threads=th) as b:
            b.step(60, dt)
            out.append(b.temperature())
    assert np.array_equal(out[0], out[1]) and np.array_equal(out[0], out[2])


def test_invalid_problem_rejected():
    p = mg.unit_cube(3)
    p.tets = p.tets.copy()
    p.tets[0, 0] = p.n_nodes          # node index out of range
    with pytest.raises(ValueError):
        ct.ThreadedBaseline(p, "fp64")
