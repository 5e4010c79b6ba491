"""Block kernel reading the conductances from L2 instead of shared memory:
bitwise the results of the default kernel, the oracle to 1e-9 K."""
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


@pytest.mark.parametrize("prec,threads", [("fp32", 256), ("fp32", 512), ("fp64", 256)])
def test_weights_l2_equals_default(fem, prec, threads):
    p = mg.random_small(81, nx=14, ny=12, nz=10, n_mat=3)
    o = oracle.OracleProblem(p)
    o.set_temperature(p.T0)
    dt = 0.9 * o.stable_dt()
    o.step(120, dt)
    out = []
    for wl2 in (0, 1):
        with fem.Mesh(p, prec, block_elems=256, threads=threads if wl2 else 0, weights_l2=wl2) as m:
            m.step(120, dt)
            out.append(m.temperature())
    assert np.array_equal(out[0], out[1])
    tol = 1e-9 if prec == "fp64" else 0.05
    assert np.abs(out[1] - o.temperature()).max() <= tol
