"""The checked build (device-side bounds checks on every shared-memory slot,
partial, mirror and node index; a failed check is reported as FEM_ECUDA)
runs the parity cases of every variant and option cleanly.  It stands in
for the memory checker, which is not available on the test machines.
Runs in a child process, because the library is chosen at import time."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import math, sys
import numpy as np
sys.path.insert(0, {root!r})
from paper_1005_3158_gb300 import build
build.build(checked=True)
import oracle
from paper_1005_3158_gb300 import fem, meshgen as mg
assert fem.LIB_PATH.endswith("libfem_checked.so")

def check(m, o, n, dt, tol):
    m.step(n, dt); o.step(n, dt)
    err = float(np.abs(m.temperature() - o.temperature()).max())   # raises on a failed check
    assert err <= tol, err

cases = 0
for prec, tol in (("fp64", 1e-9), ("fp32", 0.05)):
    for variant in ("block", "atomic", "colored"):
        p = mg.random_small(3, nx=6, ny=5, nz=4, n_mat=3)
        o = oracle.OracleProblem(p); o.set_temperature(p.T0)
        with fem.Mesh(p, prec, variant=variant, block_elems=64) as m:
            check(m, o, 40, 0.9 * o.stable_dt(), tol); cases += 1
    p = mg.cast_in_mold(n_cast=5, n_mold=8)
    p.k_tables = ((0, [300.0, 900.0], [120.0, 170.0]),)
    for form in (0, 1):
        o = oracle.OracleProblem(p); o.set_temperature(p.T0)
        if form: o.set_formulation(1)
        with fem.Mesh(p, prec, block_elems=200, formulation=form) as m:
            check(m, o, 40, 0.9 * o.stable_dt(), tol); cases += 1
probs = [mg.cast_in_mold(n_cast=3, n_mold=4), mg.random_small(4, nx=4, ny=4, nz=3)]
with fem.Batch(probs, "fp64", block_elems=64) as b:
    dts = 0.9 * b.instance_stable_dt()
    t_end = 20.0 * float(dts.min())
    b.advance(t_end)
    T = b.temperature()
    for i, q in enumerate(probs):
        o = oracle.OracleProblem(q); o.set_temperature(q.T0)
        c = max(1, math.ceil(t_end / dts[i] * (1.0 - 1e-12)))
        o.step(c, t_end / c)
        assert float(np.abs(b.instance_temperature(i, T) - o.temperature()).max()) <= 1e-9
    cases += 1
print("CHECKED_OK", cases)
"""


def test_checked_build_runs_clean():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, FEM_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-4000:])
    assert "CHECKED_OK 11" in r.stdout
