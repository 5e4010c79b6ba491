"""Pins of the oracle's right-hand side F - K T (Eqs. 4, 9, 14-22).

* Dense brute force: the global K and Robin face matrix assembled here from
  an independent derivation (barycentric solve for the gradients; edge-
  midpoint quadrature, exact for quadratics on a triangle, for the face
  mass) must reproduce the oracle's element-by-element residual.
* Patch test: a linear field gives zero residual at interior nodes and the
  consistent boundary flux at boundary nodes.
* Decomposition invariance: summing the partial residuals of any element
  partition (Eqs. 19-21) gives the global residual (Eq. 22 = Eq. 18).
"""
import numpy as np
import pytest

import oracle
from paper_1005_3158_gb300 import meshgen as mg


def _dense_system(p):
    n = p.n_nodes
    K = np.zeros((n, n))
    for e in range(p.n_tets):
        nodes = p.tets[e]
        x4 = p.xyz[nodes]
        M = np.hstack([np.ones((4, 1)), x4])
        G = np.linalg.solve(M, np.eye(4))[1:, :].T
        V = abs(np.linalg.det(M)) / 6.0
        k = p.materials[p.mat[e], 2]
        K[np.ix_(nodes, nodes)] += k * V * G @ G.T
    H = np.zeros((n, n))
    F = np.zeros(n)
    # linear shape functions on a triangle at the edge midpoints are
    # (1/2,1/2,0) and permutations; the 3-point midpoint rule (weights A/3)
    # integrates N_i N_j exactly.
    mids = np.array([[0.5, 0.5, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5]])
    for f in range(p.n_faces):
        nodes = p.faces[f]
        xa, xb, xc = p.xyz[nodes]
        A = 0.5 * np.linalg.norm(np.cross(xb - xa, xc - xa))
        Mf = sum(np.outer(w, w) for w in mids) * A / 3.0
        H[np.ix_(nodes, nodes)] += p.h[f] * Mf
        # integral of N_i is A/3
        F[nodes] += (A / 3.0) * (p.h[f] * p.t_inf[f] - p.q[f])
    return K, H, F


@pytest.mark.parametrize("seed", [0, 1, 2, 5])
def test_residual_matches_dense_assembly(seed):
    p = mg.random_small(seed, nx=4, ny=3, nz=3, n_mat=3)
    o = oracle.OracleProblem(p)
    K, H, F = _dense_system(p)
    rng = np.random.default_rng(seed)
    T = rng.uniform(300, 1000, p.n_nodes)
    R, qin = o.residual(T)
    expect = F - (K + H) @ T
    scale = np.abs(K).max() * 1000
    np.testing.assert_allclose(R, expect, rtol=0, atol=1e-12 * scale)
    # heat entering through the faces = sum of the face terms
    assert qin == pytest.approx((F - H @ T).sum(), rel=1e-10, abs=1e-9 * scale)


@pytest.mark.parametrize("ntets", [1, 5, 48])
def test_tiny_meshes_dense(ntets):
    if ntets == 1:
        xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) * 0.1
        tets = np.array([[0, 1, 2, 3]], np.int32)
    elif ntets == 5:
        # the 5-tet split of a cube (one central tet + four corners)
        c = np.array([[i, j, k] for k in (0, 1) for j in (0, 1) for i in (0, 1)], float) * 0.1
        xyz = c
        tets = np.array([[0, 1, 2, 4], [1, 3, 2, 7], [1, 4, 5, 7], [2, 4, 7, 6],
                         [1, 2, 4, 7]], np.int32)
    else:
        xyz, tets, _, _ = mg.box_grid(2, 2, 2, 0.1, 0.1, 0.1)
    n = xyz.shape[0]
    faces = np.array([tets[0, :3]], np.int32)
    p = mg.Problem(xyz=xyz, tets=tets, mat=np.zeros(len(tets), np.int32),
                   materials=np.array([mg.ALLOY]), faces=faces, h=np.array([500.0]),
                   t_inf=np.array([350.0]), q=np.array([100.0]), T0=np.full(n, 900.0))
    o = oracle.OracleProblem(p)
    K, H, F = _dense_system(p)
    T = np.linspace(400, 1000, n)
    R, _ = o.residual(T)
    np.testing.assert_allclose(R, F - (K + H) @ T, rtol=0,
                               atol=1e-12 * np.abs(K).max() * 1000)


def test_patch_test_linear_field():
    p = mg.unit_cube(6, jitter=0.15, seed=11)
    o = oracle.OracleProblem(p, faces=False)
    b = np.array([3.0, -2.0, 5.0])
    T = 500.0 + p.xyz @ b
    R, _ = o.residual(T)
    k = mg.ALLOY[2]
    x = p.xyz
    eps = 1e-9
    on_bnd = ((x < eps) | (x > 1 - eps)).any(axis=1)
    scale = k * np.linalg.norm(b) * (1.0 / 6)
    assert np.abs(R[~on_bnd]).max() <= 1e-12 * scale * 1e3
    # boundary nodes: R_i = - sum over the node's boundary faces of
    # k (b . n_out) A / 3  (Green's identity on the linear field)
    _, tets, _, flags = mg.box_grid(6, 6, 6)
    faces = mg.box_boundary_faces(p.tets, flags)
    expect = np.zeros(p.n_nodes)
    for f in faces:
        xa, xb, xc = x[f]
        nrm = np.cross(xb - xa, xc - xa)
        A = 0.5 * np.linalg.norm(nrm)
        nrm = nrm / np.linalg.norm(nrm)
        cen = (xa + xb + xc) / 3
        if np.dot(nrm, cen - 0.5) < 0:
            nrm = -nrm
        expect[f] -= k * np.dot(b, nrm) * A / 3
    np.testing.assert_allclose(R[on_bnd], expect[on_bnd], rtol=0, atol=1e-11 * scale * 1e3)


@pytest.mark.parametrize("nparts", [2, 3, 7])
def test_partition_sum_equals_global(nparts):
    p = mg.random_small(4, nx=6, ny=5, nz=4)
    o = oracle.OracleProblem(p)
    rng = np.random.default_rng(nparts)
    T = rng.uniform(300, 1000, p.n_nodes)
    R, q = o.residual(T)
    ep = rng.integers(0, nparts, p.n_tets).astype(np.int32)
    fp = rng.integers(0, nparts, p.n_faces).astype(np.int32)
    acc = np.zeros(p.n_nodes)
    qs = 0.0
    for k in range(nparts):
        Rk, qk = o.residual(T, ep, fp, k)
        acc += Rk
        qs += qk
    np.testing.assert_allclose(acc, R, rtol=0, atol=1e-9 * np.abs(R).max())
    assert qs == pytest.approx(q, rel=1e-12, abs=1e-9)
