"""Multi-rank host logic on the CPU (gloo, world size 2): ranks take disjoint
channel blocks that together cover the job, and the step statistics reduce
to the slowest rank's time and the sum of all ranks' evaluations.  The
collapse of blocks split across ranks: each rank's partial sums (from the
oracle's full cube restricted to its blocks) are merged by
``merge_collapse`` and normalised once; the result equals the one-rank
collapse over every channel triple."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2506_10526_gb300.sharding import (block_evals, blocks_of, cubes_of,  # noqa: E402
                                             merge_collapse, rank_block, reduce_step_stats)


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


def _partial_sums(num, valid, blocks):
    """Unfolded raw collapse sums and sampling of the given channel blocks from
    the oracle's per-triple numerators num [ntrip, nc, nc, nc]."""
    import numpy as np
    ntrip, nc = num.shape[0], num.shape[1]
    n2 = 2 * nc - 1
    sums = np.zeros((ntrip, n2, n2))
    nnu = np.zeros((n2, n2), np.int64)
    for b in blocks:
        for n1 in range(b[0], b[1]):
            for n2_ in range(b[2], b[3]):
                for n3 in range(b[4], b[5]):
                    if valid[n1] and valid[n2_] and valid[n3]:
                        sums[:, n1 - n3 + nc - 1, n2_ - n3 + nc - 1] += num[:, n1, n2_, n3]
                        nnu[n1 - n3 + nc - 1, n2_ - n3 + nc - 1] += 1
    return sums, nnu


def _merge_worker(rank, world, port, out):
    import numpy as np
    import oracle
    import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nt, nc = 16, 6
    edges = [1.0, 3.0, 5.0, 7.0]
    vis = synth.sky_visibilities(nt, nc, seed=77)
    flags = np.array([0, 0, 1, 0, 0, 0], np.uint8)
    res = oracle.mabs_full(vis.astype(np.complex128), edges, chan_flags=flags)
    jobs = blocks_of(nc, 4, 2)   # ragged blocks; nu3 split over ranks
    mine = [jobs[k] for k in range(rank, len(jobs), world)]
    s, c = _partial_sums(res["num"].real, flags == 0, mine)
    st, ct = torch.from_numpy(s), torch.from_numpy(c)
    merge_collapse(st, ct, world)
    if rank == 0:
        sums = oracle.fold_plane(st.numpy())
        cnt = oracle.fold_plane(ct.numpy())
        T = res["T"].astype(np.float64)
        with np.errstate(invalid="ignore", divide="ignore"):
            bbar = np.where(cnt > 0, sums / (T[:, None, None] * np.where(cnt > 0, cnt, 1)), np.nan)
        want, wcnt = oracle.collapse_fold(res["B"].real)
        out.put((bbar, want, cnt, wcnt[int(np.argmax(res["T"] > 0))], res["T"]))
    dist.barrier()
    dist.destroy_process_group()


def test_collapse_split_over_two_ranks_merges_to_the_one_rank_result():
    import numpy as np
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    mp.start_processes(_merge_worker, args=(world, _free_port(), q), nprocs=world, join=True,
                       start_method="spawn")
    bbar, want, cnt, wcnt, T = q.get(timeout=120)
    np.testing.assert_array_equal(cnt, wcnt)
    keep = T > 0
    assert np.array_equal(np.isnan(bbar[keep]), np.isnan(want[keep]))
    ok = ~np.isnan(want[keep])
    np.testing.assert_allclose(bbar[keep][ok], want[keep][ok], rtol=1e-12,
                               atol=1e-12 * np.nanmax(np.abs(want[keep])))


def test_sub_band_cubes_are_disjoint_cubes_covering_the_band():
    """cubes_of: every block is a cube (the same range on all three channels),
    the sub-bands are disjoint and cover [0, nc), the last one ragged."""
    for nc, side in [(768, 256), (20, 8), (7, 7), (5, 8)]:
        cubes = cubes_of(nc, side)
        for c in cubes:
            assert c[0:2] == c[2:4] == c[4:6] and c[0] < c[1]
        chans = [ch for c in cubes for ch in range(c[0], c[1])]
        assert chans == list(range(nc))
        assert sum(block_evals(c, 1) for c in cubes) == sum((c[1] - c[0]) ** 3 for c in cubes)
