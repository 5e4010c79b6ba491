"""Pins of the oracle's cast-mold interface (Eq. 8; sisters, Section 3).

* Closed form: two tets touching face to face without shared nodes, each at
  a uniform temperature: element terms vanish and every face node receives
  h A / 3 (T_other - T_own).
* Conservation: a matching interface (every face has an identical sister)
  with adiabatic outer walls keeps the total enthalpy to rounding.
* Composite bar with contact resistance: two bars meshed separately, Dirichlet
  ends T_L and T_R, interface coefficient h_i between them.  The steady state
  is exact for linear elements: q = (T_L - T_R) / (L1/k1 + 1/h_i + L2/k2),
  linear in each bar, a jump q / h_i at the interface.
* Sisters are the nearest faces of the other side (brute force here).
* The stable step accounts for the interface terms.
"""
import numpy as np
import pytest

import oracle
from paper_1005_3158_gb300 import meshgen as mg


def _problem(xyz, tets, mat, mats, T0, faces=None, h=None, tinf=None, ia=None, ib=None, hi=2000.0,
             dir_nodes=None, dir_T=None):
    F = np.zeros((0, 3), np.int32) if faces is None else faces
    nf = F.shape[0]
    return mg.Problem(xyz=xyz, tets=tets.astype(np.int32), mat=mat.astype(np.int32),
                      materials=np.array(mats, float), faces=F.astype(np.int32),
                      h=np.full(nf, 1000.0) if h is None else h,
                      t_inf=np.full(nf, 300.0) if tinf is None else tinf, q=np.zeros(nf),
                      T0=np.asarray(T0, float),
                      dir_nodes=np.zeros(0, np.int32) if dir_nodes is None else dir_nodes.astype(np.int32),
                      dir_T=np.zeros(0) if dir_T is None else dir_T,
                      iface_a=ia.astype(np.int32), iface_b=ib.astype(np.int32),
                      h_ia=np.full(ia.shape[0], hi), h_ib=np.full(ib.shape[0], hi))


def test_two_tets_closed_form():
    # tet A below the plane z = 0, tet B above it, their faces on z = 0
    # coincide but use separate nodes
    xyz = np.array([[0, 0, 0], [0.1, 0, 0], [0, 0.1, 0], [0, 0, -0.1],
                    [0, 0, 0], [0.1, 0, 0], [0, 0.1, 0], [0, 0, 0.1]], float)
    tets = np.array([[0, 1, 2, 3], [4, 5, 6, 7]])
    TA, TB = 900.0, 400.0
    p = _problem(xyz, tets, np.zeros(2), [mg.STEEL], [TA] * 4 + [TB] * 4,
                 ia=np.array([[0, 1, 2]]), ib=np.array([[4, 5, 6]]), hi=1500.0)
    o = oracle.OracleProblem(p)
    o.set_temperature(p.T0)
    R, qin = o.residual(o.temperature())
    A = 0.5 * 0.1 * 0.1
    expect = 1500.0 * A / 3.0
    np.testing.assert_allclose(R[[0, 1, 2]], expect * (TB - TA), rtol=1e-12)
    np.testing.assert_allclose(R[[4, 5, 6]], expect * (TA - TB), rtol=1e-12)
    np.testing.assert_allclose(R[[3, 7]], 0.0, atol=1e-9)
    assert qin == pytest.approx(0.0, abs=1e-9)
    assert list(o.interface_sisters()) == [1, 0]


def test_matching_interface_conserves_energy():
    # cast_in_mold with equal spacing on both sides: the interface matches
    p = mg.cast_in_mold(n_cast=4, n_mold=8)
    p.faces = np.zeros((0, 3), np.int32)
    p.h = p.t_inf = p.q = np.zeros(0)
    o = oracle.OracleProblem(p)
    sis = o.interface_sisters()
    na = p.iface_a.shape[0]
    assert (sis[sis] == np.arange(sis.shape[0])).all()          # mutual pairs
    assert (sis[:na] >= na).all() and (sis[na:] < na).all()      # across sides
    o.set_temperature(p.T0)
    dt = 0.9 * o.stable_dt()
    U0 = o.energy()[1]
    o.step(300, dt)
    U, _, Qb, _ = o.energy()
    assert abs(U - U0) <= 1e-12 * U0
    assert abs(Qb) <= 1e-12 * U0
    T = o.temperature()
    assert T.max() < 973.0 and T.min() > 300.0                   # heat crossed over


def _bar(nx, x0, length, w=0.02):
    xyz, tets, _, flags = mg.box_grid(nx, 1, 1, length, w, w)
    xyz = xyz + np.array([x0, 0, 0])
    lo = mg.box_boundary_faces(tets, flags, plane_mask=1)
    hi = mg.box_boundary_faces(tets, flags, plane_mask=2)
    return xyz, tets, flags, lo, hi


@pytest.mark.parametrize("n1,n2", [(6, 6), (5, 8)])
def test_composite_bar_contact_resistance(n1, n2):
    L1, L2, hi, TL, TR = 0.06, 0.04, 800.0, 900.0, 300.0
    k1, k2 = 150.0, 30.0
    xa, ta, fa, _, a_hi = _bar(n1, 0.0, L1)
    xb, tb, fb, b_lo, _ = _bar(n2, L1, L2)
    nb0 = xa.shape[0]
    xyz = np.concatenate([xa, xb])
    tets = np.concatenate([ta, tb + nb0])
    mat = np.concatenate([np.zeros(len(ta)), np.ones(len(tb))])
    mats = [(2700.0, 900.0, k1, 0, 0, 0), (7800.0, 460.0, k2, 0, 0, 0)]
    left = np.nonzero(fa & 1)[0]
    right = np.nonzero(fb & 2)[0] + nb0
    d = np.concatenate([left, right])
    dT = np.concatenate([np.full(len(left), TL), np.full(len(right), TR)])
    p = _problem(xyz, tets, mat, mats, np.full(xyz.shape[0], 600.0), ia=a_hi, ib=b_lo + nb0,
                 hi=hi, dir_nodes=d, dir_T=dT)
    o = oracle.OracleProblem(p)
    o.set_temperature(p.T0)
    dt = 0.9 * o.stable_dt()
    T_prev = o.temperature()
    for _ in range(400):
        o.step(500, dt)
        T = o.temperature()
        if np.abs(T - T_prev).max() < 1e-11:
            break
        T_prev = T
    q = (TL - TR) / (L1 / k1 + 1.0 / hi + L2 / k2)
    x = xyz[:, 0]
    exact = np.where(np.arange(xyz.shape[0]) < nb0, TL - q * x / k1,
                     TR + q * (L1 + L2 - x) / k2)
    np.testing.assert_allclose(T, exact, rtol=0, atol=1e-7)
    # the jump across the contact is q / h_i
    jump = T[np.argmin(np.where(np.arange(len(x)) < nb0, np.abs(x - L1), 9))] - \
        T[nb0 + np.argmin(np.abs(xb[:, 0] - L1))]
    assert jump == pytest.approx(q / hi, rel=1e-8)


def test_sisters_nearest_and_stable_dt():
    p = mg.cast_in_mold(n_cast=5, n_mold=8)     # non-matching
    o = oracle.OracleProblem(p)
    sis = o.interface_sisters()
    F = np.concatenate([p.iface_a, p.iface_b])
    cen = p.xyz[F].mean(axis=1)
    na = p.iface_a.shape[0]
    for f in range(0, len(F), 7):
        other = np.arange(na, len(F)) if f < na else np.arange(na)
        d = ((cen[other] - cen[f]) ** 2).sum(axis=1)
        assert sis[f] == other[np.argmin(d)]
    # the interface only adds to the Gershgorin rows: a smaller stable step
    q = mg.cast_in_mold(n_cast=5, n_mold=8)
    q.iface_a = np.zeros((0, 3), np.int32)
    q.iface_b = np.zeros((0, 3), np.int32)
    q.h_ia = q.h_ib = np.zeros(0)
    dt_if, dt_no = o.stable_dt(), oracle.OracleProblem(q).stable_dt()
    assert dt_if < dt_no
    o.set_temperature(p.T0)
    o.step(2000, 0.9 * dt_if)
    # bounded (the consistent face matrices allow small over- and undershoots
    # of the ambient temperature; no discrete maximum principle is claimed)
    T = o.temperature()
    assert np.isfinite(T).all() and T.max() <= 974.0 and T.min() >= 299.0
