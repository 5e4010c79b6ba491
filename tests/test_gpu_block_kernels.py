"""The two forms of the block kernel compute the same numbers: with
constant k and the enthalpy formulation the default (256 threads) reads
the conductances from L2, any other thread count stages them in shared
memory.  Both give bitwise the same temperatures and boundary heat, and
the FP64 oracle to 1e-9 K (FP32 0.05 K)."""
import numpy as np
import pytest

import oracle
from paper_1005_3158_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fem():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1005_3158_gb300 import fem as f
    return f


@pytest.mark.parametrize("prec,be", [("fp32", 256), ("fp32", 0), ("fp64", 200), ("fp64", 0)])
def test_l2_and_staged_conductances_agree(fem, prec, be):
    p = mg.random_small(81, nx=14, ny=12, nz=10, n_mat=3)
    o = oracle.OracleProblem(p)
    o.set_temperature(p.T0)
    dt = 0.9 * o.stable_dt()
    o.step(120, dt)
    out = []
    for threads in (0, 512):   # 0: the default, 256 threads with L2 conductances
        with fem.Mesh(p, prec, block_elems=be, threads=threads) as m:
            m.step(120, dt)
            out.append((m.temperature(), m.energy()))
            if threads == 0:
                assert m.info()["threads"] == 256
    tol = 1e-9 if prec == "fp64" else 0.05
    if be > 0 or prec == "fp64":   # the same partition: the same sums
        assert np.array_equal(out[0][0], out[1][0])
        assert out[0][1][2] == out[1][1][2]
    else:   # FP32 defaults: 1,792-tet blocks (L2) against 2,048 (staged)
        assert np.abs(out[0][0] - out[1][0]).max() <= tol
    assert np.abs(out[0][0] - o.temperature()).max() <= tol
