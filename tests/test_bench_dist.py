"""bench.py's multi-process helpers (barrier, max and sum over ranks) with two gloo ranks
on the CPU: the whole-job value is the units of all ranks over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    w, r = bench.init_dist("gloo")
    bench.barrier()
    t = bench.max_over_ranks(1.0 + rank)
    n = bench.sum_over_ranks(10.0 * (rank + 1))
    q.put((r, w, t, n))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_max_and_sum():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] == 2 and o[2] == 2.0 and o[3] == 30.0 for o in out)
