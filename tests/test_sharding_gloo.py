"""Multi-rank host logic on the CPU (gloo, world size 2): ranks take disjoint
channel blocks that together cover the job, and the step statistics reduce
to the slowest rank's time and the sum of all ranks' evaluations."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2506_10526_gb300.sharding import (block_evals, blocks_of, rank_block,  # noqa: E402
                                             reduce_step_stats)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, nc, bsz, steps, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    jobs = blocks_of(nc, bsz)
    mine = [rank_block(jobs, i, world, rank) for i in range(steps)]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    ms, evals = reduce_step_stats(10.0 + rank, sum(block_evals(b, 7) for b in mine), world)
    if rank == 0:
        out.put((gathered, ms, evals))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_disjoint_blocks_covering_the_job():
    nc, bsz, world = 12, 8, 2   # 2^3 = 8 blocks, ragged (8 + 4) along each axis
    jobs = blocks_of(nc, bsz)
    steps = len(jobs) // world
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    mp.start_processes(_worker, args=(world, _free_port(), nc, bsz, steps, q), nprocs=world,
                       join=True, start_method="spawn")
    gathered, ms, evals = q.get(timeout=60)
    assert not set(gathered[0]) & set(gathered[1])          # disjoint
    assert set(gathered[0]) | set(gathered[1]) == set(jobs)  # covering one pass of the job
    assert ms == 11.0                                         # slowest rank
    assert evals == 7 * nc ** 3                               # every channel triple once
