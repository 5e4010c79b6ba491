"""Pins of the oracle's temperature-dependent conductivity (Eq. 9 allows
K(T); reading: a piecewise-linear k(T) per material evaluated at the
element's mean temperature at step n).

* A one-point table equal to the constant k reproduces the constant-k run.
* Adiabatic walls conserve energy exactly for any k(T) (K^e(T) keeps zero
  row sums).
* Single tet: R = -k(mean T) K_unit T, with K_unit the k = 1 matrix.
* Steady bar with k = k0 + k1 T between Dirichlet ends: the Kirchhoff
  transform Phi(T) = k0 T + k1 T^2 / 2 is linear in x, which gives the exact
  profile; the element-mean-k discretisation converges to it at second
  order (error ratio ~4 per halving of h).
"""
import numpy as np
import pytest

import oracle
from paper_1005_3158_gb300 import meshgen as mg


def test_one_point_table_is_constant_k():
    p = mg.random_small(3, nx=5, ny=4, nz=4, n_mat=2)
    dt = 0.9 * oracle.OracleProblem(p).stable_dt()
    a = oracle.OracleProblem(p)
    a.set_temperature(p.T0)
    a.step(100, dt)
    b = oracle.OracleProblem(p)
    for mt in range(p.materials.shape[0]):
        b.set_conductivity(mt, [500.0], [p.materials[mt, 2]])
    assert b.stable_dt() == pytest.approx(dt / 0.9, rel=1e-12)
    b.set_temperature(p.T0)
    b.step(100, dt)
    np.testing.assert_allclose(b.temperature(), a.temperature(), rtol=0, atol=1e-9)


def test_conductivity_table_interpolation():
    p = mg.unit_cube(2)
    o = oracle.OracleProblem(p)
    o.set_conductivity(0, [300.0, 600.0, 900.0], [100.0, 160.0, 130.0])
    assert o.conductivity(0, 200.0) == 100.0
    assert o.conductivity(0, 450.0) == pytest.approx(130.0, rel=1e-15)
    assert o.conductivity(0, 750.0) == pytest.approx(145.0, rel=1e-15)
    assert o.conductivity(0, 1200.0) == 130.0
    with pytest.raises(ValueError):
        o.set_conductivity(0, [600.0, 300.0], [1.0, 2.0])     # not ascending
    with pytest.raises(ValueError):
        o.set_conductivity(0, [300.0], [-1.0])               # k <= 0


def test_adiabatic_conservation_with_k_of_T():
    p = mg.random_small(4, nx=5, ny=5, nz=4, n_mat=2)
    p.faces = np.zeros((0, 3), np.int32)
    p.h = p.t_inf = p.q = np.zeros(0)
    o = oracle.OracleProblem(p)
    for mt in range(p.materials.shape[0]):
        o.set_conductivity(mt, [300.0, 700.0, 1000.0], [20.0, 200.0, 60.0])
    o.set_temperature(p.T0)
    o.step(400, 0.9 * o.stable_dt())
    U, U0, Qb, _ = o.energy()
    assert Qb == 0.0 and abs(U - U0) <= 1e-12 * U0


def test_single_tet_closed_form():
    xyz = np.array([[0, 0, 0], [0.1, 0, 0], [0, 0.1, 0], [0, 0, 0.1]], float)
    p = mg.Problem(xyz=xyz, tets=np.array([[0, 1, 2, 3]], np.int32), mat=np.zeros(1, np.int32),
                   materials=np.array([mg.STEEL]), faces=np.zeros((0, 3), np.int32),
                   h=np.zeros(0), t_inf=np.zeros(0), q=np.zeros(0),
                   T0=np.array([400.0, 800.0, 500.0, 900.0]))
    o = oracle.OracleProblem(p)
    o.set_conductivity(0, [300.0, 1000.0], [10.0, 80.0])
    T = p.T0
    R, _ = o.residual(T)
    k = 10.0 + 70.0 * (T.mean() - 300.0) / 700.0
    # unit right tet scaled by 0.1: K = k * 0.1/6 * [[3,-1,-1,-1],[-1,1,0,0],...]
    K1 = 0.1 / 6.0 * np.array([[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]], float)
    np.testing.assert_allclose(R, -k * K1 @ T, rtol=1e-12)


def _steady_bar(n, k0, k1, TL, TR, L=0.1):
    xyz, tets, flags, _ = mg.bar(n, L)
    mats = np.array([[1000.0, 100.0, k0, 0, 0, 0]])
    d = np.concatenate([np.nonzero(flags & 1)[0], np.nonzero(flags & 2)[0]]).astype(np.int32)
    dT = np.where(xyz[d, 0] < L / 2, TL, TR)
    p = mg.Problem(xyz=xyz, tets=tets, mat=np.zeros(len(tets), np.int32), materials=mats,
                   faces=np.zeros((0, 3), np.int32), h=np.zeros(0), t_inf=np.zeros(0),
                   q=np.zeros(0), T0=np.full(xyz.shape[0], 0.5 * (TL + TR)), dir_nodes=d, dir_T=dT,
                   k_tables=((0, [0.0, 2000.0], [k0, k0 + k1 * 2000.0]),))
    o = oracle.OracleProblem(p)
    o.set_temperature(p.T0)
    dt = 0.9 * o.stable_dt()
    prev = o.temperature()
    for _ in range(2000):
        o.step(200, dt)
        T = o.temperature()
        if np.abs(T - prev).max() < 1e-12:
            break
        prev = T
    x = xyz[:, 0]
    phi = lambda t: k0 * t + 0.5 * k1 * t * t
    target = phi(TL) + (phi(TR) - phi(TL)) * x / L
    exact = (-k0 + np.sqrt(k0 * k0 + 2.0 * k1 * target)) / k1
    return np.abs(T - exact).max()


def test_kirchhoff_steady_state_second_order():
    e1 = _steady_bar(8, 20.0, 0.2, 1000.0, 300.0)
    e2 = _steady_bar(16, 20.0, 0.2, 1000.0, 300.0)
    assert e2 < 0.5            # K
    assert 3.0 < e1 / e2 < 5.0
