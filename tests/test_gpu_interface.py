"""GPU parity of the cast-mold interface (Eq. 8): a cube casting meshed on
its own inside a box mold, the two meshes meeting without matching nodes;
the CUDA path against the FP64 oracle (FP64 1e-9 K, FP32 0.05 K)."""
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
@pytest.mark.parametrize("variant", ["block", "atomic"])
def test_cast_in_mold_matches_oracle(fem, prec, variant):
    p = mg.cast_in_mold(n_cast=9, n_mold=8)
    o = oracle.OracleProblem(p)
    dt = 0.9 * o.stable_dt()
    o.set_temperature(p.T0)
    with fem.Mesh(p, prec, variant=variant, block_elems=200) as m:
        assert m.stable_dt() == pytest.approx(o.stable_dt(), rel=1e-13)
        for _ in range(5):
            m.step(100, dt)
            o.step(100, dt)
            err = np.abs(m.temperature() - o.temperature()).max()
            assert err <= TOL[prec], f"{err:.3e} K"
        U, U0, Qb, lat = m.energy()
        eo = o.energy()
        rel = 1e-12 if prec == "fp64" else 1e-5
        assert abs(U - U0 - Qb) <= rel * abs(U0)
        assert Qb == pytest.approx(eo[2], rel=1e-9 if prec == "fp64" else 1e-3)
        # heat left the casting through the interface into the mold
        T = m.temperature()
        n_mold = p.xyz.shape[0] - (9 + 1) ** 3
        assert T[n_mold:].max() < 973.0 and T[:n_mold].max() > 300.0


def test_batch_with_interfaces(fem):
    probs = [mg.cast_in_mold(n_cast=7, n_mold=8), mg.cast_in_mold(n_cast=5, n_mold=4)]
    with fem.Batch(probs, "fp64", block_elems=150) as b:
        dt = 0.9 * b.instance_stable_dt()
        t_end = 60.0 * float(dt.min())
        b.advance(t_end)
        T = b.temperature()
        for i, p in enumerate(probs):
            o = oracle.OracleProblem(p)
            assert dt[i] == pytest.approx(0.9 * o.stable_dt(), rel=1e-13)
            o.set_temperature(p.T0)
            c = max(1, math.ceil(t_end / dt[i] * (1.0 - 1e-12)))
            o.step(c, t_end / c)
            assert np.abs(b.instance_temperature(i, T) - o.temperature()).max() <= 1e-9
