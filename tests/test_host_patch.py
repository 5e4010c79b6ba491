"""The patch used by the full-size parity tests: one oracle step of the
patch around sampled nodes equals, on those nodes, one oracle step of the
whole mesh (same temperatures at step n)."""
import numpy as np

import oracle
from paper_1005_3158_gb300 import meshgen as mg
from patching import patch, sample_nodes


def test_patch_step_equals_full_step():
    p = mg.block_with_cores(14, n_cores=4)
    o = oracle.OracleProblem(p)
    o.set_temperature(p.T0)
    dt = 0.9 * o.stable_dt()
    o.step(40, dt)
    Tn = o.temperature()
    S, n_mushy = sample_nodes(p, Tn, np.random.default_rng(1), n_random=200, n_each=50)
    assert n_mushy > 0
    o.step(1, dt)
    sub, used, s_loc = patch(p, S)
    assert sub.n_tets < p.n_tets
    q = oracle.OracleProblem(sub)
    q.set_temperature(Tn[used])
    q.step(1, dt)
    assert np.abs(q.temperature()[s_loc] - o.temperature()[S]).max() <= 1e-9


def test_patch_detects_a_dropped_element():
    """A patch that misses one element of a sampled node gives that node a
    different step (so the harness would catch a kernel dropping it)."""
    p = mg.unit_cube(6)
    o = oracle.OracleProblem(p)
    o.set_temperature(p.T0)
    dt = 0.9 * o.stable_dt()
    o.step(10, dt)
    Tn = o.temperature()
    o.step(1, dt)
    S = np.array([p.tets[100, 0]])
    sub, used, s_loc = patch(p, S)
    sub.tets, sub.mat = sub.tets[1:], sub.mat[1:]
    q = oracle.OracleProblem(sub)
    q.set_temperature(Tn[used])
    q.step(1, dt)
    assert abs(q.temperature()[s_loc][0] - o.temperature()[S][0]) > 1e-6
