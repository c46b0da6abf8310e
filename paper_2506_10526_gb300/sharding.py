"""Host-side sharding of the channel cube across ranks (one process per GPU).

The job of a plan is the full channel cube nc^3 of every closable ring
triple.  It splits into blocks of B x B x B3 channels (nu1 x nu2 x nu3, the
last ones ragged; B3 = B unless given); rank r of
W takes blocks r, r + W, r + 2W, ... in step order, so ranks never share a
block and need no data-path collective: each rank's collapse sums hold its
own blocks (the sum over ranks is the job's).  Timing is the maximum over
ranks; throughput counts every rank's evaluations.

When ranks split nu3, one plane of the collapse (Section 3.2: the mean over
channel triples sharing (dnu1, dnu2)) gathers triples from several ranks:
``merge_collapse`` sums every rank's raw accumulators (bs_delta_export) and
unfolded sampling before any rank normalises (bs_delta_import, then
bs_mabs_delta / bs_bs3d).  That sum is the path's one exchange step.
"""
from __future__ import annotations


def blocks_of(nc: int, bsz: int, bsz3: int | None = None):
    """Half-open channel blocks (nu1_lo, nu1_hi, nu2_lo, nu2_hi, nu3_lo, nu3_hi):
    sides bsz along nu1 and nu2, bsz3 (default bsz) along nu3."""
    b3 = bsz if not bsz3 else bsz3
    n = (nc + bsz - 1) // bsz
    n3 = (nc + b3 - 1) // b3
    out = []
    for a in range(n):
        for b in range(n):
            for c in range(n3):
                out.append((a * bsz, min(nc, (a + 1) * bsz), b * bsz, min(nc, (b + 1) * bsz),
                            c * b3, min(nc, (c + 1) * b3)))
    return out


def cubes_of(nc: int, side: int):
    """Sub-band cubes S x S x S, S = [s, s + side) (the last one ragged), as
    blocks: the job of channel-symmetric accumulation (bs_mabs accumulate = 2),
    which takes only cubes.  Each cube is one sub-band's whole channel cube."""
    return [(s, min(nc, s + side)) * 3 for s in range(0, nc, side)]


def rank_block(jobs, step: int, world: int, rank: int):
    """Block of `rank` at `step` (steps cycle through the job)."""
    return jobs[(step * world + rank) % len(jobs)]


def block_evals(block, closable_triples: int) -> int:
    b = block
    return closable_triples * (b[1] - b[0]) * (b[3] - b[2]) * (b[5] - b[4])


def reduce_step_stats(ms: float, evals: float, world: int, device=None):
    """(max over ranks of the elapsed ms, sum over ranks of evaluations)."""
    if world <= 1:
        return ms, evals
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e = torch.tensor([float(evals)], dtype=torch.float64, device=device)
    dist.all_reduce(e)
    return float(t.item()), float(e.item())


def merge_collapse(sums, nnu, world: int):
    """Sum the partial collapse accumulators of every rank in place: ``sums``
    the raw pixel sums [batch, ntrip, 2nc-1, 2nc-1] (float64) and ``nnu`` the
    unfolded sampling [2nc-1, 2nc-1] (int64), both torch tensors on the rank's
    communication device.  Returns them; a no-op for one rank."""
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(sums)
        dist.all_reduce(nnu)
    return sums, nnu
