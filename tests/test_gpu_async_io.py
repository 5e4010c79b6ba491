"""Pipelined host I/O (fem_set_state_async / fem_get_temperature_async /
fem_sync): a host loop that uploads a different state every iteration,
steps and reads the temperatures back gives, iteration by iteration, the
bits of the same loop through the synchronous calls (the deterministic
block variant; the atomic variant to its rounding) -- whatever the overlap
of the copies with the steps."""
import numpy as np
import pytest

from paper_1005_3158_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1005_3158_gb300 import fem as f
    return f, torch


@pytest.mark.parametrize("prec,variant", [("fp32", "block"), ("fp64", "block"), ("fp32", "atomic")])
def test_async_loop_equals_sync_loop(env, prec, variant):
    fem, torch = env
    p = mg.random_small(51, nx=10, ny=9, nz=8, n_mat=3)
    n_iter = 7
    with fem.Mesh(p, prec, variant=variant) as m:
        dt = 0.9 * m.stable_dt()
        m.step(5, dt)
        E0 = m.state()[0]
        rng = np.random.default_rng(3)
        # a different state every iteration: E0 scaled by up to +-1 %
        inputs = [torch.from_numpy(E0 * rng.uniform(0.99, 1.01, E0.size)).pin_memory()
                  for _ in range(n_iter)]
        ref = []
        for k in range(n_iter):
            m.set_state(inputs[k].numpy(), k, k * dt)
            m.step(2, dt)
            ref.append(m.temperature())
        outs = [torch.empty(m.n_nodes, dtype=torch.float64).pin_memory() for _ in range(n_iter)]
        for k in range(n_iter):
            m.set_state_async(inputs[k], k, k * dt)
            m.step(2, dt)
            m.temperature_async(outs[k])
        m.sync()
        # the block variant is deterministic (bitwise); the atomic variant
        # adds in a run-dependent order (last-bit differences)
        same = np.array_equal if variant == "block" else \
            (lambda x, y: np.allclose(x, y, rtol=0, atol=1e-3))
        for k in range(n_iter):
            assert same(outs[k].numpy(), ref[k]), f"iteration {k}"
        # the state after the loop is that of the last iteration
        assert same(m.temperature(), ref[-1])


def test_async_reuses_one_host_buffer_in_order(env):
    """One pinned output buffer written by every iteration holds the last
    iteration's temperatures after fem_sync (copies stay in call order)."""
    fem, torch = env
    p = mg.unit_cube(10)
    with fem.Mesh(p, "fp32") as m:
        dt = 0.9 * m.stable_dt()
        E = torch.from_numpy(m.state()[0]).pin_memory()
        out = torch.empty(m.n_nodes, dtype=torch.float64).pin_memory()
        for k in range(5):
            m.set_state_async(E, 0, 0.0)
            m.step(k + 1, dt)
            m.temperature_async(out)
        m.sync()
        m.set_state(E.numpy(), 0, 0.0)
        m.step(5, dt)
        assert np.array_equal(out.numpy(), m.temperature())


def test_async_non_finite_state_reported_by_sync(env):
    fem, torch = env
    p = mg.unit_cube(6)
    with fem.Mesh(p, "fp64") as m:
        E = m.state()[0].copy()
        E[3] = np.nan
        m.set_state_async(E, 0, 0.0)
        with pytest.raises(fem.FemError) as e:
            m.sync()
        assert e.value.status == fem.FEM_EINVAL


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_async_f32_host_arrays(env, prec):
    """FP32 host arrays: the upload converts to the mesh's precision and
    the read-back rounds T to FP32 -- the same numbers as the FP64 calls
    (exactly the same for an FP32 mesh, whose E and T are FP32 anyway)."""
    fem, torch = env
    p = mg.random_small(52, nx=9, ny=8, nz=7, n_mat=3)
    with fem.Mesh(p, prec) as m:
        dt = 0.9 * m.stable_dt()
        m.step(5, dt)
        E32 = m.state()[0].astype(np.float32)
        m.set_state(E32.astype(np.float64), 0, 0.0)
        m.step(3, dt)
        T_ref = m.temperature()
        E_h = torch.from_numpy(E32).pin_memory()
        T_h = torch.empty(m.n_nodes, dtype=torch.float32).pin_memory()
        m.set_state_async(E_h, 0, 0.0)
        m.step(3, dt)
        m.temperature_async(T_h)
        m.sync()
        assert np.array_equal(T_h.numpy(), T_ref.astype(np.float32))
