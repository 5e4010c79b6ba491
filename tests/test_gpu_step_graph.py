"""fem_step(n) replays a captured graph of 32 steps for n >= 32 and
launches the rest directly; the results are those of single-step calls
(bitwise for the deterministic variants), also when dt changes between
calls (the graph is captured again) and for every kernel set of a step
(interface faces, flat variants, coloured launches)."""
import numpy as np
import pytest

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


def _run(fem, p, prec, variant, plan, **kw):
    with fem.Mesh(p, prec, variant=variant, **kw) as m:
        dt = 0.9 * m.stable_dt()
        for n, scale in plan:
            if n == "single":
                for _ in range(scale[0]):
                    m.step(1, dt * scale[1])
            else:
                m.step(n, dt * scale)
        return m.temperature(), m.state()[1:]


@pytest.mark.parametrize("prec,variant", [("fp32", "block"), ("fp64", "block"), ("fp64", "colored")])
def test_graph_steps_equal_single_steps(fem, prec, variant):
    p = mg.random_small(61, nx=8, ny=7, nz=6, n_mat=3)
    Tg, (sg, tg) = _run(fem, p, prec, variant, [(70, 1.0), (40, 0.5), (33, 1.0)])
    Ts, (ss, ts) = _run(fem, p, prec, variant, [("single", (70, 1.0)), ("single", (40, 0.5)),
                                                 ("single", (33, 1.0))])
    assert sg == ss == 143
    assert tg == pytest.approx(ts, rel=1e-13)
    assert np.array_equal(Tg, Ts)


def test_graph_steps_with_interface(fem):
    p = mg.cast_in_mold(n_cast=5, n_mold=4)
    Tg, _ = _run(fem, p, "fp64", "block", [(64, 1.0)])
    Ts, _ = _run(fem, p, "fp64", "block", [("single", (64, 1.0))])
    assert np.array_equal(Tg, Ts)
