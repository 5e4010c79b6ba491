"""Host-side logic of libfem, on the CPU (no GPU needed).

* The library loads and exports every symbol declared in include/fem.h.
* Argument validation returns the documented status codes.
* The block plan is consistent: every element corner and face corner is
  scheduled exactly once, to the node it belongs to; slot indices stay
  inside the block's shared-memory slots; interior nodes belong to one block;
  shared-node copy lists cover every block that touches the node.
* The library's stable step equals the oracle's (same reading of Eq. 13,
  computed by independent code).
* Reverse Cuthill-McKee reduces the bandwidth of a randomly numbered mesh.
"""
import re

import numpy as np
import pytest

import oracle
from paper_1005_3158_gb300 import meshgen as mg

fem = pytest.importorskip("paper_1005_3158_gb300.fem")

HEADER = __import__("os").path.join(__import__("os").path.dirname(__file__), "..", "include", "fem.h")


def test_exports_every_declared_symbol():
    text = open(HEADER).read()
    declared = set(re.findall(r"^(?:fem_status|const char \*|void)\s*\*?\s*(fem_\w+)\s*\(",
                              text, flags=re.M))
    assert declared, "no declarations parsed"
    assert declared == set(fem.ABI_SYMBOLS)
    for name in declared:
        assert hasattr(fem.lib(), name), name


def _mesh(p, **kw):
    return fem.Mesh(p, kw.pop("precision", "fp32"), set_temperature=False, **kw)


def test_validation_errors():
    p = mg.random_small(0, permute=False)
    bad = p.tets.copy()
    bad[3, 1] = p.n_nodes
    with pytest.raises(fem.FemError) as e:
        fem.fem_mesh_create(p.xyz, bad, p.mat)
    assert e.value.status == fem.FEM_EINVAL
    rep = p.tets.copy()
    rep[0, 1] = rep[0, 0]
    with pytest.raises(fem.FemError):
        fem.fem_mesh_create(p.xyz, rep, p.mat)
    with pytest.raises(fem.FemError):
        fem.fem_mesh_create(p.xyz, p.tets, -np.ones(p.n_tets))
    h = fem.fem_mesh_create(p.xyz, p.tets, p.mat)
    try:
        with pytest.raises(fem.FemError) as e:
            fem.fem_step(h, 1, 1.0)
        assert e.value.status == fem.FEM_ESTATE
        mats = p.materials.copy()
        mats[0, 2] = -1.0
        with pytest.raises(fem.FemError):
            fem.fem_set_materials(h, mats)
        with pytest.raises(fem.FemError):
            fem.fem_set_materials(h, p.materials[:1])     # mat id out of range
        fem.fem_set_materials(h, p.materials)
        # an interior face (shared by two tets) is not a boundary face
        t0 = p.tets[0]
        with pytest.raises(fem.FemError) as e:
            fem.fem_set_boundary(h, [t0[[0, 1, 2]], t0[[1, 2, 3]], t0[[0, 1, 3]], t0[[0, 2, 3]]],
                                 np.ones(4), np.ones(4))
        assert e.value.status == fem.FEM_EINVAL
        with pytest.raises(fem.FemError):
            fem.fem_set_boundary(h, p.faces[:1], [-1.0], [300.0])
        with pytest.raises(fem.FemError):
            fem.fem_set_temperature(h, np.full(p.n_nodes, np.nan))
        with pytest.raises(fem.FemError):
            fem.fem_step(h, -1, 1.0)
        with pytest.raises(fem.FemError):
            fem.fem_step(h, 1, 0.0)
    finally:
        fem.fem_mesh_destroy(h)


def test_degenerate_tet_rejected():
    p = mg.random_small(1, permute=False)
    xyz = p.xyz.copy()
    t0 = p.tets[0]
    xyz[t0[3]] = (xyz[t0[0]] + xyz[t0[1]] + xyz[t0[2]]) / 3
    with pytest.raises(fem.FemError) as e:
        fem.fem_mesh_create(xyz, p.tets, p.mat)
    assert "degenerate" in str(e.value)


def _check_plan(p, m):
    blocks = m.plan("blocks").reshape(-1, 16)
    sched = m.plan("sched").astype(np.int64)
    grp = m.plan("grp")
    elem_order = m.plan("elem_order")
    face_order = m.plan("face_order")
    copy_node = m.plan("copy_node")
    sh_ptr, sh_copy = m.plan("sh_ptr"), m.plan("sh_copy")
    copy_pos = m.plan("copy_pos")
    node_new = m.plan("node_new")
    node_old = np.empty_like(node_new)
    node_old[node_new] = np.arange(p.n_nodes)
    assert np.array_equal(np.sort(node_new), np.arange(p.n_nodes))
    n_int = int(blocks[:, 5].sum())
    # Robin faces, then interface faces (side A, side B)
    allf = np.concatenate([p.faces, getattr(p, "iface_a", np.zeros((0, 3), np.int32)),
                           getattr(p, "iface_b", np.zeros((0, 3), np.int32))]).astype(np.int64)
    seen_elem = np.zeros(p.n_tets, int)
    seen_face = np.zeros(allf.shape[0], int)
    touched_by = [set() for _ in range(p.n_nodes)]
    stride = max(((g + 4) // 4) * 4 + 16 * r for g, r in zip(blocks[:, 9], blocks[:, 14]))
    for b, (e0, ne, f0, nf, n0, nint, c0, nsh, g0, ngrp, ne_pad, nf_pad, nep, r0, nrounds, _) in enumerate(blocks):
        assert e0 % 8 == 0 and f0 % 8 == 0 and ne_pad >= ne and nf_pad >= nf
        assert nep % 8 == 0 and ne <= nep and e0 == b * nep   # uniform element stride
        assert grp[g0] == r0 and grp[g0 + ngrp] == r0 + nrounds
        if b + 1 < len(blocks):
            assert blocks[b + 1][0] == e0 + nep and blocks[b + 1][13] == r0 + nrounds
        # schedule chunks: header (ngrp+1 offsets padded to 4 words) + 16
        # words per round, at a fixed stride = the largest chunk
        assert blocks[b][15] == b * stride and ((ngrp + 4) // 4) * 4 + 16 * nrounds <= stride
        nslot = 4 * ne_pad + 3 * nf_pad
        assert nslot <= 65535
        nloc = nint + nsh
        assert ngrp == (nloc + 31) // 32
        local_nodes = np.concatenate([n0 + np.arange(nint), copy_node[c0:c0 + nsh]])
        assert (local_nodes[:nint] < n_int).all() and (copy_node[c0:c0 + nsh] >= n_int).all()
        slot_owner = np.full(nslot, -1)
        dummy = nslot
        for g in range(ngrp):
            ra, rb = grp[g0 + g], grp[g0 + g + 1]
            assert ra % 2 == 0 and rb % 2 == 0
            # (round r, lane) at (r/2)*64 + 2*lane + r%2
            S = sched[32 * ra:32 * rb].reshape(-1, 32, 2)
            for lane in range(32):
                l = 32 * g + lane
                col = S[:, lane, :].ravel()
                assert (col <= dummy).all()
                col = col[col != dummy]
                if l >= nloc:
                    assert col.size == 0
                    continue
                assert (col < nslot).all()
                assert (slot_owner[col] == -1).all()
                slot_owner[col] = local_nodes[l]
        # every element corner / face corner slot maps to its node
        for i in range(ne):
            e = elem_order[e0 + i]
            assert e >= 0
            seen_elem[e] += 1
            for c in range(4):
                assert slot_owner[c * ne_pad + i] == node_new[p.tets[e, c]]
                touched_by[p.tets[e, c]].add(b)
        for i in range(nf):
            f = face_order[f0 + i]
            seen_face[f] += 1
            for c in range(3):
                assert slot_owner[4 * ne_pad + c * nf_pad + i] == node_new[allf[f, c]]
        # padding slots are never scheduled
        used = np.zeros(nslot, bool)
        for c in range(4):
            used[c * ne_pad:c * ne_pad + ne] = True
        for c in range(3):
            used[4 * ne_pad + c * nf_pad:4 * ne_pad + c * nf_pad + nf] = True
        assert ((slot_owner >= 0) == used).all()
    assert (seen_elem == 1).all() and (seen_face == 1).all()
    # interior nodes are touched by one block, shared nodes by all their copies
    for n in range(p.n_nodes):
        i = node_new[n]
        if i < n_int:
            assert len(touched_by[n]) == 1
        else:
            s = i - n_int
            copies = sh_copy[sh_ptr[s]:sh_ptr[s + 1]]
            assert len(copies) == len(touched_by[n]) >= 2
            assert (copy_node[copies] == i).all()
            assert (copy_pos[copies] == np.arange(sh_ptr[s], sh_ptr[s + 1])).all()


@pytest.mark.parametrize("seed,block_elems", [(0, 64), (3, 100), (5, 333), (7, 5000)])
def test_block_plan_invariants(seed, block_elems):
    p = mg.random_small(seed, nx=7, ny=6, nz=5, n_mat=3)
    with _mesh(p, block_elems=block_elems) as m:
        _check_plan(p, m)
        info = m.info()
        assert info["n_interior_nodes"] + info["n_shared_nodes"] == p.n_nodes
        assert info["max_block_elems"] <= max(block_elems, 64)


def test_block_plan_unit_cube():
    p = mg.unit_cube(8)
    with _mesh(p, block_elems=256) as m:
        _check_plan(p, m)


@pytest.mark.parametrize("seed", range(4))
def test_stable_dt_matches_oracle(seed):
    p = mg.random_small(seed, n_mat=3)
    with _mesh(p, precision="fp64") as m:
        assert m.stable_dt() == pytest.approx(oracle.OracleProblem(p).stable_dt(), rel=1e-12)


def test_stable_dt_with_dirichlet():
    p = mg.random_small(8)
    p.dir_nodes = np.arange(0, p.n_nodes, 7, dtype=np.int32)
    p.dir_T = np.full(p.dir_nodes.size, 500.0)
    with _mesh(p, precision="fp64") as m:
        assert m.stable_dt() == pytest.approx(oracle.OracleProblem(p).stable_dt(), rel=1e-12)


def test_rcm_reduces_bandwidth():
    p = mg.permute_nodes(mg.unit_cube(10), mg.rng_of(3))
    perm, before, after = fem.fem_rcm_order(p.n_nodes, p.tets)
    assert np.array_equal(np.sort(perm), np.arange(p.n_nodes))
    assert after < before / 5
    # natural grid numbering of a 10^3 cube has bandwidth 11*11+11+1 = 133;
    # RCM of the shuffled mesh must be in the same range
    assert after <= 2 * 133


def test_flat_plans():
    p = mg.random_small(2, nx=6, ny=5, nz=4)
    for variant in ("atomic", "colored"):
        with _mesh(p, variant=variant) as m:
            info = m.info()
            order = m.plan("elem_order")
            valid = order[order >= 0]
            assert np.array_equal(np.sort(valid), np.arange(p.n_tets))
            if variant == "colored":
                assert 4 <= info["n_colors"] <= 64
