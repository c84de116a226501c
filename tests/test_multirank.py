"""The N > 1 path of bench.py (independent replicas, one per GPU) reduces
per-rank timings with MAX and work with SUM.  Checked here with two gloo
ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as tdist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    secs, cw = bench.reduce_over_ranks(tdist, 1.0 + rank, 1000 * (rank + 1),
                                                     torch.device("cpu"))
    q.put((rank, secs, cw))
    tdist.barrier()
    tdist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, secs, cw in out:
        assert secs == 2.0      # the slowest replica
        assert cw == 3000.0     # every replica's work
