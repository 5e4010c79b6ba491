"""GPU parity of the temperature-dependent conductivity k(T) (Eq. 9's K(T),
evaluated at each element's mean temperature of step n) against the FP64
oracle (FP64 1e-9 K, FP32 0.05 K), block and atomic variants, and in a
batch."""
import math

import numpy as np
import pytest

import oracle
from paper_1005_3158_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 0.05}
TABLES = ((0, [300.0, 600.0, 900.0, 1000.0], [60.0, 190.0, 120.0, 90.0]),
          (1, [300.0, 1000.0], [25.0, 40.0]))


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
@pytest.mark.parametrize("variant,block_elems", [("block", 96), ("block", 2048), ("atomic", 0)])
def test_k_of_T_matches_oracle(fem, prec, variant, block_elems):
    p = mg.random_small(8, nx=8, ny=6, nz=5, n_mat=3)
    p.k_tables = TABLES
    o = oracle.OracleProblem(p)
    dt = 0.9 * o.stable_dt()
    o.set_temperature(p.T0)
    with fem.Mesh(p, prec, variant=variant, block_elems=block_elems) as m:
        for _ in range(4):
            m.step(50, dt)
            o.step(50, dt)
            err = np.abs(m.temperature() - o.temperature()).max()
            assert err <= TOL[prec], f"{err:.3e} K"
        U, U0, Qb, _ = m.energy()
        assert abs(U - U0 - Qb) <= (1e-12 if prec == "fp64" else 1e-5) * abs(U0)


def test_k_of_T_casting_and_batch(fem):
    probs = [mg.flanged_casting(12, 12, 12, seed=3), mg.cast_in_mold(n_cast=5, n_mold=8)]
    for p in probs:
        p.k_tables = TABLES
    with fem.Batch(probs, "fp64", block_elems=300) as b:
        dt = 0.9 * b.instance_stable_dt()
        t_end = 40.0 * float(dt.min())
        b.advance(t_end)
        T = b.temperature()
        for i, p in enumerate(probs):
            o = oracle.OracleProblem(p)
            assert dt[i] == pytest.approx(0.9 * o.stable_dt(), rel=1e-13)
            o.set_temperature(p.T0)
            c = max(1, math.ceil(t_end / dt[i] * (1.0 - 1e-12)))
            o.step(c, t_end / c)
            assert np.abs(b.instance_temperature(i, T) - o.temperature()).max() <= 1e-9
