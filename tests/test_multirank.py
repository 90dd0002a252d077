"""The N > 1 path of bench.py on CPU: two gloo ranks.  Each rank solves its
own projection (distinct seeds, no data exchange); the job's time is the
slowest rank's and the rate counts every rank's projection."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank                  # rank 1 is the slower one
    m = bench.max_over_ranks(ms, world)
    out[rank] = (m, bench.whole_job_rate(m, world, 2048 * 2048), bench.rank_seed(rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0                     # max over ranks
    assert abs(res[0][1] - 2 / 0.015) < 1e-9                  # both ranks' projections
    assert res[0][2] != res[1][2]                             # distinct projections
