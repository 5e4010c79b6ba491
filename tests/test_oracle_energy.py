"""Energy pins of the oracle's explicit step (Eqs. 4, 14, 22).

* Adiabatic walls: the total enthalpy is conserved (column sums of every
  K^e vanish) to rounding over 1000 steps.
* Robin walls, uniform initial T0: the first step changes the energy by
  exactly -dt h A_total (T0 - T_inf) (the consistent face matrix has row
  sums h A / 3; the load is h A T_inf / 3 per corner).
* Uniform T0 = T_inf with no flux stays uniform.
* The cumulative boundary heat balances the enthalpy change.
"""
import numpy as np
import pytest

import oracle
from paper_1005_3158_gb300 import meshgen as mg


def test_adiabatic_conservation():
    p = mg.random_small(7, nx=6, ny=5, nz=4, n_mat=2)
    o = oracle.OracleProblem(p, faces=False)
    o.set_temperature(p.T0)
    dt = 0.9 * o.stable_dt()
    U0 = o.energy()[0]
    o.step(1000, dt)
    U = o.energy()[0]
    assert abs(U - U0) <= 1e-12 * abs(U0)
    # and the field really evolved
    assert np.abs(o.temperature() - p.T0).max() > 10.0


def test_first_step_robin_energy_unit_cube():
    p = mg.unit_cube(20)
    o = oracle.OracleProblem(p)
    o.set_temperature(p.T0)
    dt = 0.9 * o.stable_dt()
    e0 = o.energy()
    o.step(1, dt)
    e1 = o.energy()
    expect = -dt * mg.H_AMB * 6.0 * (mg.T_POUR - mg.T_AMB)
    assert e1[0] - e0[0] == pytest.approx(expect, rel=1e-9)
    assert e1[2] == pytest.approx(expect, rel=1e-12)


def test_uniform_equilibrium_stays_uniform():
    p = mg.random_small(3, nx=5, ny=5, nz=5)
    p.t_inf = np.full(p.n_faces, 650.0)
    p.q = np.zeros(p.n_faces)
    o = oracle.OracleProblem(p)
    o.set_temperature(np.full(p.n_nodes, 650.0))
    o.step(500, 0.9 * o.stable_dt())
    assert np.abs(o.temperature() - 650.0).max() < 1e-9


@pytest.mark.parametrize("seed", [0, 9])
def test_energy_balance_with_robin(seed):
    p = mg.random_small(seed, nx=6, ny=4, nz=4)
    o = oracle.OracleProblem(p)
    o.set_temperature(p.T0)
    o.step(700, 0.9 * o.stable_dt())
    U, U0, Qb, lat = o.energy()
    assert abs(U - U0 - Qb) <= 1e-11 * abs(U0)
    C, _, Lc = o.lumped()
    assert 0.0 <= lat <= Lc.sum() * (1 + 1e-12)
