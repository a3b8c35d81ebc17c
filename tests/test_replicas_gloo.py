"""The N > 1 path of bench.py on CPU: two gloo ranks.

The solve does not shard here (one GPU per box, independent right-hand sides
per rank), so the multi-rank logic is: distinct right-hand sides per rank,
the job's time is the slowest rank's, and the reported value is seconds per
solve over all ranks.  No data-path collective exists to test.
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
