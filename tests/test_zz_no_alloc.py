"""GPU test of fem_energy_sums_noalloc, the entry point that allocates nothing.

Callers that cannot call cudaMalloc (code running during CUDA-graph
capture, real-time loops with a no-allocation rule, processes whose device
memory belongs to another allocator) hand the library device arrays they
already own; the entry point keeps its per-CTA partial sums (one pair per
8192 nodes) in a static device array inside the library.  Its sums are
checked, on two calls in a row, against

* the energy account of the mesh API (fem_get_energy) for a stepped state,
* the FP64 oracle's energy of the same state, at sizes that take one CTA,
  several CTAs with a ragged tail, and an exact multiple of 8192 nodes,
* the oracle on a mesh with two phase-change ranges, where the phase byte
  selects the range (its high bit set on some nodes, which must be ignored),

with the tolerances of the other energy tests (FP64 1e-12 relative, FP32
1e-6 relative), plus, for the latent sum, the rounding of T(E) in the
working precision (see _check).  The two calls must agree bit for bit.

The file is named to be collected last, so a run that stops at the first
failure has run every other test first.
"""
import numpy as np
import pytest

import oracle
from paper_1005_3158_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu

REL = {"fp64": 1e-12, "fp32": 1e-6}
NODES_PER_CTA = 8192


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1005_3158_gb300 import fem
    return torch, fem


def _phase_of(p):
    """Per node: index of its phase-change range in the sorted range list,
    and that list (each node touches at most one phase-change material)."""
    ranges = sorted({(m[4], m[5]) for m in p.materials if m[3] > 0}) or [(0.0, 0.0)]
    ph = np.zeros(p.n_nodes, np.uint8)
    for mt, m in enumerate(p.materials):
        if m[3] > 0:
            ph[p.tets[p.mat == mt].ravel()] = ranges.index((m[4], m[5]))
    return ph, ranges


def _device_state(torch, p, E, prec, ph=None):
    """Device copies of the state and of the node data the sums need."""
    dtype = torch.float64 if prec == "fp64" else torch.float32
    C, _, Lc = oracle.OracleProblem(p).lumped()
    ph0, ranges = _phase_of(p)
    ph = ph0 if ph is None else ph
    dev = torch.device("cuda")
    return (torch.tensor(E, dtype=dtype, device=dev), torch.tensor(C, dtype=dtype, device=dev),
            torch.tensor(Lc, dtype=dtype, device=dev), torch.tensor(ph, device=dev),
            torch.tensor(np.array(ranges).ravel(), dtype=dtype, device=dev))


def _sums_twice(torch, fem, prec, dev_state, n):
    Ed, Cd, Lcd, phd, rgd = dev_state
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    code = fem.FEM_FP64 if prec == "fp64" else fem.FEM_FP32
    results = []
    for _ in range(2):
        out.fill_(float("nan"))
        fem.fem_energy_sums_noalloc(code, Ed.data_ptr(), Cd.data_ptr(), Lcd.data_ptr(),
                                    phd.data_ptr(), rgd.data_ptr(), n, out.data_ptr(), stream)
        torch.cuda.synchronize()
        results.append(out.cpu().numpy().copy())
    assert np.array_equal(results[0], results[1])
    return results


def _check(results, U_ref, lat_ref, prec, C_sum, T_max=1000.0):
    """The latent sum E - C T(E) of a rounded state carries, per node, the
    rounding of T(E) in the working precision (a few ulps of T, worth C_i
    ulp(T) joules) even where the exact latent heat is zero: the absolute
    tolerance is 4 u T_max sum C_i, u the unit roundoff."""
    u = 2.0 ** -24 if prec == "fp32" else 2.0 ** -53
    for U, lat in results:
        assert U == pytest.approx(U_ref, rel=REL[prec])
        assert lat == pytest.approx(lat_ref, rel=REL[prec], abs=4 * u * T_max * C_sum)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["unit_cube", "random"])
def test_matches_mesh_energy_two_calls(env, prec, case):
    torch, fem = env
    p = mg.unit_cube(12) if case == "unit_cube" else mg.random_small(3, nx=8, ny=7, nz=6)
    with fem.Mesh(p, prec, reorder=1) as m:
        dt = 0.9 * m.stable_dt()
        m.step(150, dt)
        ref = m.energy()                    # U, U0, boundary heat, latent
        E = m.state()[0]
    results = _sums_twice(torch, fem, prec, _device_state(torch, p, E, prec), p.n_nodes)
    C_sum = oracle.OracleProblem(p).lumped()[0].sum()
    _check(results, ref[0], ref[3], prec, C_sum)
    # the same state's energy from the oracle
    o = oracle.OracleProblem(p)
    o.set_enthalpy(E)
    ref_o = o.energy()
    _check(results, ref_o[0], ref_o[3], prec, C_sum)


def _box(nx, ny, nz):
    """One alloy box, all faces adiabatic, seeded temperatures across the
    solid, mushy and liquid ranges."""
    xyz, tets, _, _ = mg.box_grid(nx, ny, nz, jitter=0.1, seed=77)
    n = xyz.shape[0]
    T0 = mg.rng_of(78).uniform(700.0, 1000.0, size=n)
    return mg.Problem(xyz=xyz, tets=tets, mat=np.zeros(tets.shape[0], np.int32),
                      materials=np.array([mg.ALLOY]), faces=np.zeros((0, 3), np.int32),
                      h=np.zeros(0), t_inf=np.zeros(0), q=np.zeros(0), T0=T0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dims", [(24, 24, 24), (15, 31, 31), (40, 40, 40)],
                         ids=["2ctas_ragged", "2ctas_exact", "9ctas_ragged"])
def test_multi_cta_against_oracle(env, prec, dims):
    torch, fem = env
    p = _box(*dims)
    n = p.n_nodes
    n_ctas = -(-n // NODES_PER_CTA)
    assert n_ctas >= 2
    if dims == (15, 31, 31):
        assert n % NODES_PER_CTA == 0
    else:
        assert n % NODES_PER_CTA != 0
    o = oracle.OracleProblem(p)
    o.set_temperature(p.T0)
    E = o.enthalpy()
    ref = o.energy()
    results = _sums_twice(torch, fem, prec, _device_state(torch, p, E, prec), n)
    _check(results, ref[0], ref[3], prec, o.lumped()[0].sum())


def _two_ranges():
    """Two alloys with different (Ts, Tl) separated by a steel layer, so no
    node touches both phase-change materials."""
    xyz, tets, _, _ = mg.box_grid(24, 8, 8, lx=3.0, jitter=0.1, seed=79)
    cx = mg.centroids(xyz, tets)[:, 0]
    mat = np.where(cx < 1.0, 0, np.where(cx < 2.0, 2, 1)).astype(np.int32)
    alloy_b = (2500.0, 1000.0, 120.0, 3.0e5, 700.0, 760.0)
    T0 = mg.rng_of(80).uniform(650.0, 950.0, size=xyz.shape[0])
    return mg.Problem(xyz=xyz, tets=tets, mat=mat,
                      materials=np.array([mg.ALLOY, alloy_b, mg.STEEL]),
                      faces=np.zeros((0, 3), np.int32), h=np.zeros(0), t_inf=np.zeros(0),
                      q=np.zeros(0), T0=T0)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_phase_byte_selects_the_range(env, prec):
    torch, fem = env
    p = _two_ranges()
    ph, ranges = _phase_of(p)
    assert len(ranges) == 2 and (ph == 1).any() and (ph == 0).any()
    ph = ph | np.where(mg.rng_of(81).random(p.n_nodes) < 0.5, 0x80, 0).astype(np.uint8)
    o = oracle.OracleProblem(p)
    o.set_temperature(p.T0)
    E = o.enthalpy()
    ref = o.energy()
    results = _sums_twice(torch, fem, prec, _device_state(torch, p, E, prec, ph), p.n_nodes)
    _check(results, ref[0], ref[3], prec, o.lumped()[0].sum())
    # the wrong range for every node of the second alloy changes the latent sum
    wrong = _sums_twice(torch, fem, prec, _device_state(torch, p, E, prec, ph & 0x80),
                        p.n_nodes)
    assert abs(wrong[0][1] - ref[3]) > 1e-3 * ref[3]


def test_rejects_sizes_beyond_the_scratch(env):
    torch, fem = env
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    ph = torch.zeros(16, dtype=torch.uint8, device="cuda")
    for n in (0, -5, 134217728 + 1):
        with pytest.raises(fem.FemError) as e:
            fem.fem_energy_sums_noalloc(fem.FEM_FP64, buf.data_ptr(), buf.data_ptr(),
                                        buf.data_ptr(), ph.data_ptr(), buf.data_ptr(), n,
                                        buf.data_ptr())
        assert e.value.status == fem.FEM_EINVAL
        assert "static scratch" in str(e.value)
    with pytest.raises(fem.FemError):
        fem.fem_energy_sums_noalloc(fem.FEM_FP64, 0, buf.data_ptr(), buf.data_ptr(),
                                    ph.data_ptr(), buf.data_ptr(), 16, buf.data_ptr())
