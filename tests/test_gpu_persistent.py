"""The persistent block kernel (fem_options.persistent: one CTA per SM that
double-buffers its element blocks) computes every block exactly as the
one-CTA-per-block kernel does: bitwise the same results, the FP64 oracle to
1e-9 K, in batches too, and it rejects what it does not support."""
import math

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


@pytest.mark.parametrize("prec,threads,be", [("fp64", 1024, 64), ("fp32", 1024, 128),
                                             ("fp32", 512, 96), ("fp64", 0, 0)])
def test_persistent_equals_block_kernel(fem, prec, threads, be):
    # 34,560 tets: with 64-128-tet blocks every CTA of the persistent grid
    # (one per SM) walks through several blocks and both of its buffers
    p = mg.random_small(71, nx=20, ny=18, nz=16, n_mat=3)
    o = oracle.OracleProblem(p)
    o.set_temperature(p.T0)
    dt = 0.9 * o.stable_dt()
    o.step(150, dt)
    out = []
    for persistent in (0, 1):
        with fem.Mesh(p, prec, block_elems=be, threads=threads if persistent else 0,
                      persistent=persistent) as m:
            m.step(150, dt)
            out.append((m.temperature(), m.energy()))
            if persistent:
                assert m.info()["ctas_per_sm"] == 1
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1][2] == out[1][1][2]   # boundary heat, same per-block order
    tol = 1e-9 if prec == "fp64" else 0.05
    assert np.abs(out[1][0] - o.temperature()).max() <= tol


def test_persistent_batch_advance(fem):
    probs = [mg.random_small(s, nx=nx, ny=ny, nz=nz, n_mat=2)
             for s, (nx, ny, nz) in zip([72, 73, 74], [(6, 5, 4), (4, 4, 4), (7, 5, 5)])]
    # a batch takes the options of its parts: build it from persistent parts
    parts = [fem.Mesh(p, "fp64", block_elems=64, persistent=1) for p in probs]
    try:
        h = fem.fem_batch_create([q.h for q in parts])
    finally:
        for q in parts:
            q.close()
    try:
        dt = fem.fem_instance_stable_dt(h, len(probs)) * 0.9
        t_end = 20.0 * float(dt.min())
        fem.fem_advance(h, t_end)
        n = sum(p.n_nodes for p in probs)
        T = fem.fem_get_temperature(h, n)
        start = np.cumsum([0] + [p.n_nodes for p in probs])
        for i, p in enumerate(probs):
            o = oracle.OracleProblem(p)
            o.set_temperature(p.T0)
            c = max(1, math.ceil(t_end / dt[i] * (1.0 - 1e-12)))
            o.step(c, t_end / c)
            assert np.abs(T[start[i]:start[i + 1]] - o.temperature()).max() <= 1e-9
    finally:
        fem.fem_mesh_destroy(h)


def test_persistent_rejections(fem):
    p = mg.unit_cube(4)
    with pytest.raises(fem.FemError):
        fem.Mesh(p, "fp32", variant="atomic", persistent=1)
    with fem.Mesh(p, "fp32", persistent=1, threads=256) as m:
        with pytest.raises(fem.FemError) as e:
            m.step(1, 1e-3)
        assert e.value.status == fem.FEM_EINVAL
