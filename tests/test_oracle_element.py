"""Pins of the oracle's element matrix and lumped capacities (Section 3).

K^e of the linear tet is pinned to (a) the closed form of the unit right tet
and (b) an independent derivation through the barycentric coefficient matrix
[1 x y z]^{-1} (numpy solve), plus its invariants.  Lumping is pinned to the
totals rho c V, rho V and rho L V_alloy that row-sum lumping must preserve.
"""
import numpy as np
import pytest

import oracle
from paper_1005_3158_gb300 import meshgen as mg


def _shape_gradients_barycentric(x4):
    """grad N_j from the inverse of M = [1 x y z] (rows = corners): the
    coefficients of N_j are column j of M^{-1}."""
    M = np.hstack([np.ones((4, 1)), x4])
    coef = np.linalg.solve(M, np.eye(4))
    return coef[1:, :].T, abs(np.linalg.det(M)) / 6.0   # [4,3], |V|


def test_unit_right_tet_closed_form():
    # corners (0,0,0),(1,0,0),(0,1,0),(0,0,1): V = 1/6, gradients
    # (-1,-1,-1), e_x, e_y, e_z, so K = k/6 [[3,-1,-1,-1],[-1,1,0,0],...]
    x = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    k = 7.0
    K, V = oracle.tet_matrix(x, k)
    expect = k / 6.0 * np.array([[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0],
                                 [-1, 0, 0, 1]], float)
    assert V == pytest.approx(1.0 / 6.0, rel=1e-15)
    np.testing.assert_allclose(K, expect, rtol=0, atol=1e-14)


def test_negative_orientation_volume_sign():
    x = np.array([[0, 0, 0], [1, 0, 0], [0, 0, 1], [0, 1, 0]], float)
    K, V = oracle.tet_matrix(x, 1.0)
    assert V == pytest.approx(-1.0 / 6.0)
    # the matrix uses |V| and is the same as the positively oriented one
    # with corners 2 and 3 exchanged
    K2, _ = oracle.tet_matrix(x[[0, 1, 3, 2]], 1.0)
    np.testing.assert_allclose(K, K2[[0, 1, 3, 2]][:, [0, 1, 3, 2]], atol=1e-15)


@pytest.mark.parametrize("seed", range(8))
def test_random_tet_against_barycentric(seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(4, 3))
    k = rng.uniform(1, 200)
    K, V = oracle.tet_matrix(x, k)
    G, absV = _shape_gradients_barycentric(x)
    expect = k * absV * G @ G.T
    assert abs(V) == pytest.approx(absV, rel=1e-12)
    np.testing.assert_allclose(K, expect, rtol=1e-10, atol=1e-12 * np.abs(expect).max())
    # symmetric, zero row sums, PSD with one zero eigenvalue
    np.testing.assert_allclose(K, K.T, atol=1e-12 * np.abs(K).max())
    np.testing.assert_allclose(K.sum(axis=1), 0, atol=1e-12 * np.abs(K).max())
    ev = np.linalg.eigvalsh(K)
    assert ev[0] > -1e-10 * ev[-1] and abs(ev[0]) < 1e-10 * ev[-1] and ev[1] > 0


def test_rigid_motion_and_scaling():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(4, 3))
    K, _ = oracle.tet_matrix(x, 3.0)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    xr = x @ Q.T + rng.normal(size=3)
    Kr, _ = oracle.tet_matrix(xr, 3.0)
    np.testing.assert_allclose(Kr, K, atol=1e-12 * np.abs(K).max())
    s = 2.5
    Ks, _ = oracle.tet_matrix(s * x, 3.0)      # k V |grad N|^2 scales as s
    np.testing.assert_allclose(Ks, s * K, rtol=1e-12, atol=1e-13)


def test_lumped_totals_unit_cube():
    p = mg.unit_cube(20)
    o = oracle.OracleProblem(p)
    C, m, Lc = o.lumped()
    rho, c, k, L, Ts, Tl = mg.ALLOY
    assert C.sum() == pytest.approx(rho * c * 1.0, rel=1e-13)   # 2.43e6 J/K
    assert m.sum() == pytest.approx(rho * 1.0, rel=1e-13)
    assert Lc.sum() == pytest.approx(rho * L * 1.0, rel=1e-13)
    assert (C > 0).all() and (m > 0).all()
    # interior node of the Kuhn grid: 24 tets of volume h^3/6 around it
    hsz = 1.0 / 20
    n_int = 10 + 21 * (10 + 21 * 10)
    assert C[n_int] == pytest.approx(rho * c * hsz ** 3, rel=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_lumped_totals_two_materials(seed):
    p = mg.random_small(seed, n_mat=3)
    o = oracle.OracleProblem(p)
    C, m, Lc = o.lumped()
    x, t = p.xyz, p.tets
    vol = np.abs(np.linalg.det(np.stack([x[t[:, 1]] - x[t[:, 0]], x[t[:, 2]] - x[t[:, 0]],
                                         x[t[:, 3]] - x[t[:, 0]]], axis=2))) / 6
    M = p.materials[p.mat]
    assert C.sum() == pytest.approx((M[:, 0] * M[:, 1] * vol).sum(), rel=1e-12)
    assert m.sum() == pytest.approx((M[:, 0] * vol).sum(), rel=1e-12)
    assert Lc.sum() == pytest.approx((M[:, 0] * M[:, 3] * vol).sum(), rel=1e-12)
    assert vol.sum() == pytest.approx(np.prod(x.max(0) - x.min(0)), rel=1e-12)


def test_degenerate_tet_rejected():
    p = mg.random_small(1, permute=False)
    p.xyz = p.xyz.copy()
    t0 = p.tets[0]
    # collapse corner 3 onto the plane of corners 0,1,2 (tet volume 0)
    p.xyz[t0[3]] = (p.xyz[t0[0]] + p.xyz[t0[1]] + p.xyz[t0[2]]) / 3
    with pytest.raises(ValueError):
        oracle.OracleProblem(p)


def test_conflicting_phase_ranges_rejected():
    p = mg.random_small(2, n_mat=3, permute=False)
    mats = p.materials.copy()
    mats[2, 4] += 10.0          # material 2 keeps latent heat, new range
    p.materials = mats
    if not ((p.mat == 0).any() and (p.mat == 2).any()):
        pytest.skip("seed without both phase-change materials")
    with pytest.raises(ValueError):
        oracle.OracleProblem(p)
