"""The CUDA path against the hand-worked one-tet example in tests/golden/
(every variant; FP64 to 1e-9 K, FP32 to 1e-3 K on values of 300-700 K)."""
import numpy as np
import pytest

from golden_example import load, problem, vec

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 1e-3}


@pytest.fixture(scope="module")
def fem():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1005_3158_gb300 import fem as f
    return f


@pytest.mark.parametrize("variant", ["block", "atomic", "colored"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["sensible", "latent"])
def test_worked_example(fem, case, prec, variant):
    kv = load()
    p = problem(kv, case)
    with fem.Mesh(p, prec, variant=variant) as m:
        assert m.stable_dt() == pytest.approx(float(kv["dt_stable"]), rel=1e-14)
        m.step(1, float(kv["dt"]))
        err = np.abs(m.temperature() - vec(kv[f"{case}_T1"])).max()
        assert err <= TOL[prec], f"{err:.3e} K"
        U, U0, Qb, lat = m.energy()
        eU, eU0, eQ, eL = vec(kv[f"{case}_energy"])
        tol = 1e-9 if prec == "fp64" else 1e-3
        assert (U, U0, Qb, lat) == pytest.approx((eU, eU0, eQ, eL), abs=tol)
