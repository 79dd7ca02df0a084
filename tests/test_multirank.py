"""The N > 1 host path of bench.py on CPU: two gloo ranks, each timing its own
independent system; the job's time is the slowest rank and its work the sum
(weak scaling, no data-path collective)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, units = bench.reduce_over_ranks(10.0 + 5.0 * rank, 1000 * (rank + 1))
    q.put((rank, ms, units, bench.dist_env()))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_max_time_and_sum_of_units():
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
    for rank, ms, units, env in out:
        assert ms == 15.0 and units == 3000
        assert env[0] == 2 and env[1] == rank


def test_single_process_is_identity():
    import bench
    assert bench.reduce_over_ranks(3.5, 7) == (3.5, 7)
