"""Library interface (Eq. 8) on the host: the sister of every interface
face, the stable step and the plan agree with the oracle's own search and
bound (no GPU)."""
import numpy as np
import pytest

import oracle
from paper_1005_3158_gb300 import meshgen as mg

fem = pytest.importorskip("paper_1005_3158_gb300.fem")

from test_host_plan import _check_plan  # noqa: E402


@pytest.mark.parametrize("nc,nm", [(5, 8), (4, 8), (7, 12), (3, 4)])
@pytest.mark.parametrize("variant", ["block", "atomic"])
def test_sisters_and_stable_dt_match_oracle(nc, nm, variant):
    p = mg.cast_in_mold(n_cast=nc, n_mold=nm)
    o = oracle.OracleProblem(p)
    with fem.Mesh(p, "fp64", variant=variant, block_elems=128) as m:
        assert np.array_equal(m.plan("if_sister"), o.interface_sisters())
        assert m.stable_dt() == pytest.approx(o.stable_dt(), rel=1e-13)
        info = m.info()
        assert info["n_faces"] == p.faces.shape[0]
        assert info["n_interface_faces"] == p.iface_a.shape[0] + p.iface_b.shape[0]
        if variant == "block":
            _check_plan(p, m)


def test_interface_validation():
    p = mg.cast_in_mold(n_cast=3, n_mold=4)
    with fem.Mesh(p, "fp64") as m:
        a, b = p.iface_a, p.iface_b
        ha, hb = p.h_ia, p.h_ib
        with pytest.raises(fem.FemError):
            fem.fem_set_interface(m.h, a, ha, np.zeros((0, 3)), np.zeros(0))   # one side empty
        bad = a.copy()
        bad[0] = [0, 1, 2] if not {0, 1, 2} <= set(a[0]) else [0, 1, 3]
        with pytest.raises(fem.FemError):
            fem.fem_set_interface(m.h, np.array([[0, 1, 9999]]), ha[:1], b, hb)   # id out of range
        with pytest.raises(fem.FemError):
            fem.fem_set_interface(m.h, a, -ha, b, hb)                           # negative h
        # removing the interface gives the plain mesh's stable step
        fem.fem_set_interface(m.h, np.zeros((0, 3)), np.zeros(0), np.zeros((0, 3)), np.zeros(0))
        q = mg.cast_in_mold(n_cast=3, n_mold=4)
        q.iface_a = q.iface_b = np.zeros((0, 3), np.int32)
        q.h_ia = q.h_ib = np.zeros(0)
        assert m.stable_dt() == pytest.approx(oracle.OracleProblem(q).stable_dt(), rel=1e-13)
        assert m.info()["n_interface_faces"] == 0


def test_conductivity_tables_stable_dt_matches_oracle():
    p = mg.random_small(6, nx=5, ny=4, nz=4, n_mat=3)
    p.k_tables = ((0, [300.0, 600.0, 1000.0], [20.0, 180.0, 90.0]), (2, [500.0], [7.0]))
    o = oracle.OracleProblem(p)
    for variant in ("block", "atomic"):
        with fem.Mesh(p, "fp64", variant=variant) as m:
            assert m.stable_dt() == pytest.approx(o.stable_dt(), rel=1e-13)
    with fem.Mesh(p, "fp64") as m:
        with pytest.raises(fem.FemError):
            fem.fem_set_conductivity(m.h, 5, [300.0], [1.0])            # no material 5
        with pytest.raises(fem.FemError):
            fem.fem_set_conductivity(m.h, 0, [600.0, 300.0], [1.0, 2.0])  # not ascending
        with pytest.raises(fem.FemError):
            fem.fem_set_conductivity(m.h, 0, [300.0], [0.0])             # k <= 0


def test_formulation_validation():
    p = mg.unit_cube(3)
    with pytest.raises(fem.FemError):
        fem.Mesh(p, "fp64", variant="atomic", formulation="apparent")
    q = mg.unit_cube(3)
    q.materials = np.array([[2700.0, 900.0, 150.0, 3.9e5, 933.0, 933.0]])
    with pytest.raises(fem.FemError):
        fem.Mesh(q, "fp64", formulation="apparent")
    with fem.Mesh(p, "fp64", formulation="apparent") as m:
        assert m.stable_dt() == pytest.approx(oracle.OracleProblem(p).stable_dt(), rel=1e-13)
