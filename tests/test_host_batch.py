"""Batches of independent meshes: host-side plan and validation (no GPU).

A batch is the disjoint union of its parts; its plan must satisfy every
invariant of a single mesh's plan (checked on the concatenated problem) and,
in addition, keep every element block inside one instance, with the
instances' blocks contiguous and ordered by stable step (smallest first).
"""
import numpy as np
import pytest

from paper_1005_3158_gb300 import meshgen as mg

fem = pytest.importorskip("paper_1005_3158_gb300.fem")

from test_host_plan import _check_plan  # noqa: E402


def _parts(seeds, sizes):
    return [mg.random_small(s, nx=nx, ny=ny, nz=nz, n_mat=2) for s, (nx, ny, nz) in zip(seeds, sizes)]


@pytest.mark.parametrize("precision,block_elems", [("fp64", 64), ("fp32", 100)])
def test_batch_plan_invariants(precision, block_elems):
    probs = _parts([1, 2, 3, 4], [(4, 3, 3), (6, 5, 4), (3, 3, 3), (5, 4, 4)])
    cat = mg.concat_problems(probs)
    with fem.Batch(probs, precision, block_elems=block_elems) as b:
        _check_plan(cat, b)
        info = b.info()
        assert info["n_instances"] == 4
        block_inst = b.plan("block_inst")
        start = b.plan("inst_block_start")
        order = b.plan("inst_order")
        blocks = b.plan("blocks").reshape(-1, 16)
        elem_order = b.plan("elem_order")
        es = np.cumsum([0] + [p.n_tets for p in probs])
        # blocks of plan position k belong to instance order[k], contiguously
        assert start[0] == 0 and start[-1] == len(blocks)
        for k, i in enumerate(order):
            assert (block_inst[start[k]:start[k + 1]] == i).all()
            assert start[k + 1] - start[k] == -(-probs[i].n_tets // block_elems)
            for bl in range(start[k], start[k + 1]):
                e0, ne = blocks[bl][0], blocks[bl][1]
                els = elem_order[e0:e0 + ne]
                assert ((els >= es[i]) & (els < es[i + 1])).all()
        # per-instance stable steps are the parts' own; plan order by them
        stable = b.instance_stable_dt()
        for i, p in enumerate(probs):
            with fem.Mesh(p, precision) as m:
                assert stable[i] == pytest.approx(m.stable_dt(), rel=1e-15)
        assert (np.diff(stable[order]) >= 0).all()
        t, n = b.instance_times()
        assert (t == 0).all() and (n == 0).all()


def test_batch_validation():
    probs = _parts([5, 6], [(3, 3, 3), (4, 3, 3)])
    a = fem.Mesh(probs[0], "fp64")
    c = fem.Mesh(probs[1], "fp32")
    d = fem.Mesh(probs[1], "fp64", set_temperature=False)
    try:
        with pytest.raises(fem.FemError) as e:
            fem.fem_batch_create([a.h, c.h])
        assert e.value.status == fem.FEM_EINVAL
        with pytest.raises(fem.FemError) as e:
            fem.fem_batch_create([a.h, d.h])
        assert e.value.status == fem.FEM_ESTATE
        h = fem.fem_batch_create([a.h, a.h])   # the same part twice is two instances
        try:
            with pytest.raises(fem.FemError) as e:
                fem.fem_set_materials(h, probs[0].materials)
            assert e.value.status == fem.FEM_ESTATE
            with pytest.raises(fem.FemError) as e:
                fem.fem_batch_create([h])
            assert e.value.status == fem.FEM_EINVAL
            with pytest.raises(fem.FemError) as e:
                fem.fem_set_instance_dt(h, [1.0, -1.0])
            assert e.value.status == fem.FEM_EINVAL
            assert fem.fem_mesh_info(h)["n_nodes"] == 2 * probs[0].n_nodes
        finally:
            fem.fem_mesh_destroy(h)
        # a plain mesh is not a batch
        with pytest.raises(fem.FemError) as e:
            fem.fem_advance(a.h, 1.0)
        assert e.value.status == fem.FEM_ESTATE
    finally:
        a.close()
        c.close()
        d.close()


def test_casting_instances_recipe():
    b = mg.batched_castings(8, seed=3, lo=2e4, hi=5e4)
    n = np.array([p.n_tets for p in b])
    assert ((n > 1.0e4) & (n < 1.0e5)).all()
    for p in b:
        assert set(np.unique(p.mat)) == {0, 1}
        assert p.faces.shape[0] > 0 and (p.T0 >= 300).all()
