"""The N > 1 path of bench.py on CPU: two gloo ranks.

The solve does not shard here (one GPU per box, independent right-hand sides
per rank), so the multi-rank logic is: distinct right-hand sides per rank,
the job's time is the slowest rank's, and the reported value is seconds per
solve over all ranks.  No data-path collective exists to test.  The second
test runs that logic with real per-rank work: every rank solves its own
right-hand side (bench.replica_rhs_seed) on a small lattice with the FP64
oracle, and the ranks' systems, solutions and the job's value are checked.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    elapsed = 1.0 + 0.5 * rank                      # a slower rank 1
    m = bench.max_over_ranks(elapsed, ws, "cpu")
    seeds = [None] * ws
    dist.all_gather_object(seeds, bench.replica_rhs_seed(rank))
    out[rank] = (m, seeds, bench.whole_job_value(m, 3, ws))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas():
    ws, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        m, seeds, value = res[rank]
        assert m == 1.5                              # max over ranks
        assert len(set(seeds)) == ws                 # every rank its own rhs
        assert abs(value - 1.5 / 6) < 1e-12          # 3 solves on each of 2 ranks


def _solve_worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import time

    import numpy as np

    import bench
    import oracle
    from paper_1706_05843_gb300 import inputs as I
    dims, Ls = (2, 2, 2, 4), 4
    o = oracle.Oracle(oracle.Action(dims=dims, Ls=Ls, **bench.WORKLOAD["action"]), I.gauge_field(dims, 0.5, 1))
    phi = I.gaussian_fermion(dims, Ls, bench.replica_rhs_seed(rank))
    steps = 2
    dist.barrier()
    t0 = time.perf_counter()
    for _ in range(steps):
        psi, st = o.solve_h(phi, tol=1e-10)
    elapsed = time.perf_counter() - t0
    m = bench.max_over_ranks(elapsed, ws, "cpu")
    res = float(np.linalg.norm(phi - o.hsys(psi)) / np.linalg.norm(phi))
    norms = [None] * ws
    dist.all_gather_object(norms, (float(np.linalg.norm(phi)), float(np.linalg.norm(psi))))
    out[rank] = (elapsed, m, res, norms, bench.whole_job_value(m, steps, ws))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_solve_their_own_systems():
    import oracle
    oracle.build()  # compiled once, before the ranks start
    ws, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_solve_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    slowest = max(res[r][0] for r in range(ws))
    for rank in range(ws):
        elapsed, m, r, norms, value = res[rank]
        assert m == slowest                          # every rank reports the slowest rank's time
        assert r <= 1e-10                            # each rank's own system, solved
        assert norms[0] != norms[1]                  # distinct right-hand sides and solutions
        assert abs(value - slowest / (2 * ws)) <= 1e-15 * slowest   # solves of all ranks
