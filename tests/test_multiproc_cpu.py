"""Multi-process logic on CPU (gloo, world size 2).

* The benchmark's job-level reduction: the slowest rank's time is the job's
  time, and whole-job throughput counts every rank's units.
* The exchange a multi-GPU partition of the mesh would need (Eqs. 19-22):
  each rank assembles the residual of its own elements and faces only; the
  sum of the ranks' partial residuals (an all-reduce) equals the global
  residual, and the explicit update made from it on each rank equals the
  single-process oracle step.
"""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

import oracle
from paper_1005_3158_gb300 import meshgen as mg

WORLD = 2


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(target, *args):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=target, args=(r, WORLD, port, q) + args) for r in range(WORLD)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out, key=lambda x: x[0])


def _init(rank, world, port):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _bench_worker(rank, world, port, q):
    import bench
    dist = _init(rank, world, port)
    ms = 10.0 + 5.0 * rank            # the ranks' own timings differ
    t = bench.max_over_ranks(ms, world, "cpu")
    v = bench.job_throughput(1000, 3, world, t / 1e3)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, v))


def test_bench_reduction_takes_slowest_rank():
    out = _run(_bench_worker)
    for rank, t, v in out:
        assert t == 15.0
        assert v == pytest.approx(1000 * 3 * 2 / 0.015)


def _partition(p):
    """Two element parts by centroid x (a plane cut, as a coordinate
    bisection would make); each face goes with the tet that owns it."""
    cx = p.xyz[p.tets].mean(axis=1)[:, 0]
    ep = (cx > np.median(cx)).astype(np.int32)
    faces = np.sort(p.faces, axis=1)
    owner = {}
    for e, t in enumerate(p.tets):
        for drop in range(4):
            owner[tuple(sorted(np.delete(t, drop)))] = e
    fp = np.array([ep[owner[tuple(f)]] for f in faces], np.int32)
    return ep, fp


def _exchange_worker(rank, world, port, q, seed):
    import torch
    dist = _init(rank, world, port)
    p = mg.random_small(seed, nx=6, ny=5, nz=4, n_mat=2)
    o = oracle.OracleProblem(p, dirichlet=False)
    o.set_temperature(p.T0)
    dt = 0.9 * o.stable_dt()
    ep, fp = _partition(p)
    T = o.temperature()
    R_part, q_part = o.residual(T, ep, fp, rank)
    # Eq. 22: shared nodes receive the other part's contributions
    R = torch.from_numpy(R_part.copy())
    dist.all_reduce(R, op=dist.ReduceOp.SUM)
    qin = torch.tensor([q_part], dtype=torch.float64)
    dist.all_reduce(qin, op=dist.ReduceOp.SUM)
    E_next = o.enthalpy() + dt * R.numpy()
    dist.destroy_process_group()
    q.put((rank, R.numpy(), float(qin.item()), E_next, dt))


@pytest.mark.parametrize("seed", [0, 3])
def test_partition_exchange_equals_global_step(seed):
    oracle.build()
    out = _run(_exchange_worker, seed)
    p = mg.random_small(seed, nx=6, ny=5, nz=4, n_mat=2)
    o = oracle.OracleProblem(p, dirichlet=False)
    o.set_temperature(p.T0)
    R, qin = o.residual(o.temperature())
    scale = np.abs(R).max()
    o.step(1, out[0][4])
    for rank, R_sum, q_sum, E_next, dt in out:
        np.testing.assert_allclose(R_sum, R, rtol=0, atol=1e-12 * scale)
        assert q_sum == pytest.approx(qin, rel=1e-12, abs=1e-9)
        np.testing.assert_allclose(E_next, o.enthalpy(), rtol=1e-13)
    # both ranks hold the same state after the exchange
    np.testing.assert_array_equal(out[0][3], out[1][3])
