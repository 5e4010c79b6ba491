"""The oracle against the hand-worked one-tet example in tests/golden/
(stiffness of Eq. 9, lumped capacity, Robin face of Eq. 4, T(E) of Eqs. 5
and 11 across the mushy range, the stable step of Eq. 13 as read, and the
energy account): every value is exact, so the tolerance is rounding only."""
import numpy as np
import pytest

import oracle
from golden_example import load, problem, vec


@pytest.mark.parametrize("case", ["sensible", "latent"])
def test_worked_example(case):
    kv = load()
    p = problem(kv, case)
    o = oracle.OracleProblem(p)
    o.set_temperature(p.T0)
    assert o.stable_dt() == pytest.approx(float(kv["dt_stable"]), rel=1e-14)
    o.step(1, float(kv["dt"]))
    np.testing.assert_allclose(o.temperature(), vec(kv[f"{case}_T1"]), rtol=0, atol=1e-11)
    U, U0, Qb, lat = o.energy()
    eU, eU0, eQ, eL = vec(kv[f"{case}_energy"])
    assert (U, U0, Qb) == pytest.approx((eU, eU0, eQ), abs=1e-10)
    assert lat == pytest.approx(eL, abs=1e-10)
