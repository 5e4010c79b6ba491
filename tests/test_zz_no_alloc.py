"""GPU test of fem_energy_sums_noalloc, the entry point that allocates nothing.

Callers that cannot call cudaMalloc (code running during CUDA-graph
capture, real-time loops with a no-allocation rule, processes whose device
memory belongs to another allocator) hand the library device arrays they
already own; the entry point keeps its per-CTA partial sums in a static
device array inside the library.  Here its sums of a stepped state are
checked, on two calls in a row, against the energy account that the mesh
API (fem_get_energy) reports for the same state, with the tolerances of the
other energy tests (FP64 1e-12 relative, FP32 1e-6 relative).

The file is named to be collected last, so a run that stops at the first
failure has run every other test first.
"""
import numpy as np
import pytest

import oracle
from paper_1005_3158_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu

REL = {"fp64": 1e-12, "fp32": 1e-6}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1005_3158_gb300 import fem
    return torch, fem


def _device_state(torch, p, E, prec):
    """Device copies of the state and of the node data the sums need."""
    dtype = torch.float64 if prec == "fp64" else torch.float32
    C, _, Lc = oracle.OracleProblem(p).lumped()
    ranges = sorted({(m[4], m[5]) for m in p.materials if m[3] > 0}) or [(0.0, 0.0)]
    assert len(ranges) == 1          # the problems below have one phase-change range
    dev = torch.device("cuda")
    return (torch.tensor(E, dtype=dtype, device=dev), torch.tensor(C, dtype=dtype, device=dev),
            torch.tensor(Lc, dtype=dtype, device=dev),
            torch.zeros(p.n_nodes, dtype=torch.uint8, device=dev),
            torch.tensor(np.array(ranges).ravel(), dtype=dtype, device=dev))


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
    Ed, Cd, Lcd, phd, rgd = _device_state(torch, p, E, prec)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    code = fem.FEM_FP64 if prec == "fp64" else fem.FEM_FP32
    results = []
    for _ in range(2):
        out.fill_(float("nan"))
        fem.fem_energy_sums_noalloc(code, Ed.data_ptr(), Cd.data_ptr(), Lcd.data_ptr(),
                                    phd.data_ptr(), rgd.data_ptr(), p.n_nodes, out.data_ptr(),
                                    stream)
        torch.cuda.synchronize()
        results.append(out.cpu().numpy().copy())
    for U, lat in results:
        assert U == pytest.approx(ref[0], rel=REL[prec])
        assert lat == pytest.approx(ref[3], rel=REL[prec], abs=1e-9 * abs(ref[0]))
    assert np.array_equal(results[0], results[1])


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
