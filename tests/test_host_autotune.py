"""fem_autotune argument checks that need no GPU (they come before any
device work)."""
import numpy as np
import pytest

from paper_1005_3158_gb300 import meshgen as mg

fem = pytest.importorskip("paper_1005_3158_gb300.fem")


@pytest.mark.parametrize("be,th,steps,dt", [
    ([], None, 5, 1.0),                 # no candidate
    ([32], None, 5, 1.0),               # block too small
    ([20000], None, 5, 1.0),            # block too large
    ([512], [384], 5, 1.0),             # unsupported CTA size
    ([512], None, 0, 1.0),              # no timed step
    ([512], None, 5, -1.0),             # dt <= 0
    ([512], None, 5, float("nan")),     # dt not finite
    (list(range(64, 64 + 65)), None, 5, 1.0),   # more than 64 candidates
])
def test_autotune_rejects_bad_arguments(be, th, steps, dt):
    p = mg.unit_cube(3)
    with fem.Mesh(p, "fp32") as m:
        with pytest.raises(fem.FemError) as e:
            fem.fem_autotune(m.h, np.array(be, np.int32), th, steps, dt)
        assert e.value.status == fem.FEM_EINVAL


def test_autotune_needs_block_variant():
    p = mg.unit_cube(3)
    with fem.Mesh(p, "fp32", variant="atomic") as m:
        with pytest.raises(fem.FemError) as e:
            m.autotune([256, 512], dt=1.0)
        assert e.value.status == fem.FEM_ESTATE


def test_async_io_argument_checks():
    """The asynchronous I/O calls reject NULL buffers and a mesh without a
    state before any device work."""
    import ctypes
    p = mg.unit_cube(3)
    with fem.Mesh(p, "fp32", set_temperature=False) as m:
        assert fem.lib().fem_set_state_async(m.h, None, 0, 0.0) == fem.FEM_EINVAL
        assert fem.lib().fem_get_temperature_async(m.h, None) == fem.FEM_EINVAL
        assert fem.lib().fem_set_state_async_f32(m.h, None, 0, 0.0) == fem.FEM_EINVAL
        assert fem.lib().fem_get_temperature_async_f32(m.h, None) == fem.FEM_EINVAL
        buf = np.zeros(m.n_nodes)
        st = fem.lib().fem_get_temperature_async(m.h, ctypes.c_void_p(buf.ctypes.data))
        assert st == fem.FEM_ESTATE
        assert fem.lib().fem_sync(None) == fem.FEM_EINVAL
        assert fem.lib().fem_sync(m.h) == fem.FEM_OK   # nothing on the device yet
