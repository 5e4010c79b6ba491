"""GPU error paths of the C ABI, all raised without faulting the GPU.

* A non-finite enthalpy given to fem_set_state is detected on the device and
  reported (FEM_EINVAL) by the next synchronising call; the flag is then
  cleared and a valid state steps normally again.
* A step far above the stable limit blows the state up; fem_get_temperature
  reports FEM_EUNSTABLE (the output is still written).
* A step a little above the true limit is caught earlier, by the energy
  balance check of fem_get_energy, while every value is still finite.
* Device allocation failure, injected on the host (FEM_FAULT_ALLOC_AFTER=k
  fails every device allocation after the k-th of a mesh upload), returns
  FEM_ENOMEM from the first call that needs the device, releases the partial
  upload, and leaves the library usable.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_1005_3158_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fem():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1005_3158_gb300 import fem as f
    return f


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("variant", ["block", "atomic"])
def test_non_finite_state_reported_by_next_get(fem, prec, variant):
    p = mg.unit_cube(6)
    o = oracle.OracleProblem(p)
    dt = 0.9 * o.stable_dt()
    with fem.Mesh(p, prec, reorder=1, variant=variant, block_elems=128) as m:
        m.step(3, dt)
        E, step, t = m.state()
        bad = E.copy()
        bad[len(bad) // 2] = np.nan
        m.set_state(bad, step, t)          # asynchronous: no error yet
        with pytest.raises(fem.FemError) as ei:
            m.temperature()
        assert ei.value.status == fem.FEM_EINVAL
        # the flag was cleared; a valid state steps on normally
        m.set_state(E, step, t)
        m.step(5, dt)
        o.set_temperature(p.T0)
        o.step(8, dt)
        tol = 1e-9 if prec == "fp64" else 0.05
        assert np.abs(m.temperature() - o.temperature()).max() <= tol


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_unstable_step_reported(fem, prec):
    p = mg.unit_cube(6)
    o = oracle.OracleProblem(p)
    dt = 50.0 * o.stable_dt()
    with fem.Mesh(p, prec, reorder=1, block_elems=128) as m:
        m.step(400, dt)
        with pytest.raises(fem.FemError) as ei:
            m.temperature()
        assert ei.value.status == fem.FEM_EUNSTABLE
        # reported once; the next read reports it again because the state
        # is still non-finite
        with pytest.raises(fem.FemError):
            m.temperature()


def _lambda_max(p):
    """Largest eigenvalue of C^-1 (K + H) of a sensible-only problem, from
    the oracle's residual map applied to unit vectors."""
    o = oracle.OracleProblem(p)
    C, _, _ = o.lumped()
    n = p.n_nodes
    R0, _ = o.residual(np.zeros(n))
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = -(o.residual(e)[0] - R0)
    s = 1.0 / np.sqrt(C)
    return np.linalg.eigvalsh(s[:, None] * M * s[None, :]).max()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_energy_residual_reported_before_overflow(fem, prec):
    """At 1.2 x the true stability limit 2 / lambda_max an oscillating mode
    grows by |1 - 2.4| = 1.4 per step.  The scheme still conserves energy
    exactly, but the rounding of ever larger nodal values pushes the balance
    residual U - U0 - Q_b past its rounding bound: fem_get_energy reports
    FEM_EUNSTABLE while every temperature is still finite."""
    p = mg.unit_cube(5)
    mats = p.materials.copy()
    mats[:, 3] = 0.0
    p.materials = mats
    dt = 1.2 * 2.0 / _lambda_max(p)
    with fem.Mesh(p, prec, reorder=1, block_elems=128) as m:
        # below the limit the balance holds over many steps
        m.step(2000, 0.95 * 2.0 / _lambda_max(p))
        m.energy()
        m.set_temperature(p.T0)
        for k in range(1, 600):
            m.step(2, dt)
            try:
                m.energy()
            except fem.FemError as e:
                assert e.status == fem.FEM_EUNSTABLE
                assert "balance" in str(e)
                break
        else:
            pytest.fail("no FEM_EUNSTABLE from the energy balance")
        T = m.temperature()        # raises FEM_EUNSTABLE if anything is non-finite
        assert np.isfinite(T).all()
        assert np.abs(T - 300.0).max() > 1e3    # the state has clearly blown up
        print(f"{prec}: balance check tripped after {2 * k} steps, max |T| = "
              f"{np.abs(T).max():.3g} K")


_CHILD = r"""
import os, sys
import numpy as np
import torch
sys.path.insert(0, {root!r})
from paper_1005_3158_gb300 import fem, meshgen as mg
p = mg.unit_cube(8)

def run():
    with fem.Mesh(p, {prec!r}, reorder=1, variant={variant!r}, block_elems=128) as m:
        try:
            m.step(1, 1e-3)
            return 0, m.temperature()
        except fem.FemError as e:
            return e.status, None

status0, T0 = run()                   # loads the kernels; no injection yet
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
os.environ["FEM_FAULT_ALLOC_AFTER"] = "{k}"
status, _ = run()
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
del os.environ["FEM_FAULT_ALLOC_AFTER"]
status2, T2 = run()
print("RESULT", status0, status, free0 - free1, status2, int(np.array_equal(T0, T2)))
"""


@pytest.mark.parametrize("variant", ["block", "atomic"])
@pytest.mark.parametrize("k", [0, 1, 3, 7, 12])
def test_injected_allocation_failure(fem, variant, k):
    code = _CHILD.format(root=ROOT, prec="fp32", variant=variant, k=k)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("RESULT")][-1]
    status0, status, leaked, status2, same = map(int, line.split()[1:])
    assert status0 == 0 and status2 == 0 and same == 1
    # every upload makes more than 12 device allocations
    assert status == fem.FEM_ENOMEM
    # everything the failed upload allocated was released
    assert leaked <= 0


def test_bounded_wait_gives_up(fem, monkeypatch):
    """The block kernel's waits on its bulk copies are bounded: with the
    conductance copy announced but never issued (test hook), every CTA gives
    up after its time limit, sets the device flag and exits; the next read
    reports FEM_ETIMEOUT and the CUDA context stays usable."""
    p = mg.unit_cube(6)
    o = oracle.OracleProblem(p)
    dt = 0.9 * o.stable_dt()
    monkeypatch.setenv("FEM_FAULT_SKIP_WEIGHT_COPY", "1")
    # both forms of the block kernel: conductances from L2 (default) and
    # staged in shared memory (512 threads)
    for threads, n in ((0, 1), (512, 1)):
        with fem.Mesh(p, "fp32", reorder=1, block_elems=128, threads=threads) as m:
            m.step(n, dt)
            with pytest.raises(fem.FemError) as ei:
                m.temperature()
            assert ei.value.status == fem.FEM_ETIMEOUT
    monkeypatch.delenv("FEM_FAULT_SKIP_WEIGHT_COPY")
    with fem.Mesh(p, "fp32", reorder=1, block_elems=128) as m:
        m.step(10, dt)
        o.set_temperature(p.T0)
        o.step(10, dt)
        assert np.abs(m.temperature() - o.temperature()).max() <= 0.05


def test_torch_caching_allocator(fem):
    """Device memory through fem_set_allocator from PyTorch's caching
    allocator: the same results bit for bit, the memory shows in torch's
    accounting while the mesh lives and returns to it afterwards."""
    import torch
    p = mg.unit_cube(8)
    dt = 0.9 * oracle.OracleProblem(p).stable_dt()
    with fem.Mesh(p, "fp32") as m:
        m.step(30, dt)
        T_ref = m.temperature()
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    with fem.Mesh(p, "fp32", allocator="torch") as m:
        m.step(30, dt)
        T = m.temperature()
        held = torch.cuda.memory_allocated() - before
        assert held >= m.info()["device_bytes"]
        with pytest.raises(fem.FemError) as ei:   # too late once on the device
            fem.fem_set_allocator(m.h, None, None)
        assert ei.value.status == fem.FEM_ESTATE
    assert np.array_equal(T, T_ref)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before
