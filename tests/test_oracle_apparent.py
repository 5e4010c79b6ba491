"""Pins of the oracle's apparent-heat-capacity formulation (Eqs. 6-7,
Lemmon's method; T is the unknown, C_app lumped from each element's
apparent specific heat).

* Without latent heat the apparent specific heat is c and the formulation
  reproduces the enthalpy formulation.
* Closed forms of Eq. 7 on one element: all nodes in the mushy range (H
  linear in T) -> c + L / (Tl - Ts); all solid or all liquid -> c; uniform
  T -> dH/dT at that temperature.
* cp_app >= c for any nodal temperatures (H - c T is non-decreasing).
* On a solidifying bar both formulations approximate the same physics:
  within 1 K of each other after the mushy zone has passed, while the
  apparent-capacity form does not conserve energy exactly (the effect the
  paper's introduction names) and the enthalpy form does.
"""
import numpy as np
import pytest

import oracle
from paper_1005_3158_gb300 import meshgen as mg

C, L, TS, TL = mg.ALLOY[1], mg.ALLOY[3], mg.ALLOY[4], mg.ALLOY[5]


def _one_tet(T):
    xyz = np.array([[0, 0, 0], [0.05, 0.01, 0], [0.01, 0.06, 0.005], [0.0, 0.01, 0.04]], float)
    p = mg.Problem(xyz=xyz, tets=np.array([[0, 1, 2, 3]], np.int32), mat=np.zeros(1, np.int32),
                   materials=np.array([mg.ALLOY]), faces=np.zeros((0, 3), np.int32),
                   h=np.zeros(0), t_inf=np.zeros(0), q=np.zeros(0), T0=np.asarray(T, float))
    o = oracle.OracleProblem(p)
    o.set_temperature(p.T0)
    o.set_formulation(1)
    return o


def test_apparent_cp_closed_forms():
    mushy = [830.0, 900.0, 850.0, 870.0]
    assert _one_tet(mushy).apparent_cp(0, mushy) == pytest.approx(C + L / (TL - TS), rel=1e-12)
    solid = [400.0, 700.0, 500.0, 810.0]
    assert _one_tet(solid).apparent_cp(0, solid) == pytest.approx(C, rel=1e-12)
    liquid = [920.0, 973.0, 950.0, 1000.0]
    assert _one_tet(liquid).apparent_cp(0, liquid) == pytest.approx(C, rel=1e-12)
    assert _one_tet([860.0] * 4).apparent_cp(0, [860.0] * 4) == pytest.approx(C + L / (TL - TS))
    assert _one_tet([700.0] * 4).apparent_cp(0, [700.0] * 4) == C
    # straddling the solidus: between the two
    mixed = [700.0, 880.0, 800.0, 850.0]
    cp = _one_tet(mixed).apparent_cp(0, mixed)
    assert C < cp < C + L / (TL - TS)


def test_apparent_cp_at_least_c():
    rng = np.random.default_rng(5)
    o = _one_tet([700.0] * 4)
    for _ in range(200):
        T = rng.uniform(700.0, 1000.0, 4)
        assert o.apparent_cp(0, T) >= C * (1.0 - 1e-12)


def test_no_latent_heat_equals_enthalpy_form():
    p = mg.random_small(2, nx=5, ny=4, nz=4, n_mat=2)
    p.materials = p.materials.copy()
    p.materials[:, 3] = 0.0
    a = oracle.OracleProblem(p)
    a.set_temperature(p.T0)
    b = oracle.OracleProblem(p)
    b.set_temperature(p.T0)
    b.set_formulation(1)
    dt = 0.9 * a.stable_dt()
    a.step(200, dt)
    b.step(200, dt)
    np.testing.assert_allclose(b.temperature(), a.temperature(), rtol=0, atol=1e-9)


def test_isothermal_range_rejected():
    p = mg.unit_cube(2)
    p.materials = np.array([[2700.0, 900.0, 150.0, 3.9e5, 933.0, 933.0]])
    o = oracle.OracleProblem(p)
    with pytest.raises(ValueError):
        o.set_formulation(1)


def test_solidifying_bar_against_enthalpy_form():
    xyz, tets, flags, mats = mg.bar(40, 0.4)
    faces = mg.box_boundary_faces(tets, flags, plane_mask=1)
    p = mg.Problem(xyz=xyz, tets=tets, mat=np.zeros(len(tets), np.int32), materials=mats,
                   faces=faces, h=np.full(len(faces), 1000.0), t_inf=np.full(len(faces), 300.0),
                   q=np.zeros(len(faces)), T0=np.full(len(xyz), 973.0))
    a = oracle.OracleProblem(p)
    a.set_temperature(p.T0)
    b = oracle.OracleProblem(p)
    b.set_temperature(p.T0)
    b.set_formulation(1)
    dt = 0.5 * a.stable_dt()
    n = int(1500.0 / dt)
    a.step(n, dt)
    b.step(n, dt)
    Ta, Tb = a.temperature(), b.temperature()
    assert Ta.min() < TS and Ta.max() > TS          # the mushy zone is inside the bar
    assert np.abs(Ta - Tb).max() < 1.0
    ea, eb = a.energy(), b.energy()
    assert abs(ea[0] - ea[1] - ea[2]) < 1e-12 * ea[1]
    err_b = abs(eb[0] - eb[1] - eb[2]) / eb[1]
    assert 1e-6 < err_b < 1e-2
