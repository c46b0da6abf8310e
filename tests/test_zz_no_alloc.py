"""bs_counts_noalloc, the entry point for callers that cannot allocate device
memory (their memory belongs to a pre-allocated pool, or they must not touch
the CUDA allocator): its counts must equal those of bs_counts (the plan path)
exactly, on two calls in a row.  The second call uses a different grid and
ring layout, so stale contents of the shared static scratch would show.
Collected last so that a failure here comes after every other test."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _plan_counts(nt, edges, ngrid=None):
    import torch
    import paper_2506_10526_gb300 as bs
    plan = bs.Plan(nt, 2, edges)
    vis = torch.from_numpy(synth.sky_visibilities(nt, 2, seed=3)[None]).cuda()
    plan.grid_load(vis, ngrid=ngrid)
    tri, _ = plan.counts()
    plan.close()
    return tri


def test_counts_noalloc_matches_plan_counts_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_10526_gb300 as bs
    cases = []
    e1 = synth.edges_log(20, 4.41, 128.0)
    cases.append((256, e1, None))
    r = synth.rng(5)
    ng = r.integers(0, 3, size=(40, 40)).astype(np.float32)
    ng[1:, 1:] = np.maximum(ng[1:, 1:], ng[1:, 1:][::-1, ::-1])
    cases.append((40, synth.edges_linear(6, 20.0), torch.from_numpy(ng).cuda()))
    for nt, edges, ngrid in cases:
        nb = len(edges) - 1
        out = torch.full((nb * (nb + 1) * (nb + 2) // 6,), -7, dtype=torch.int64, device="cuda")
        bs.counts_noalloc(nt, edges, out, ngrid=ngrid)
        torch.cuda.synchronize()
        want = _plan_counts(nt, edges, ngrid)
        np.testing.assert_array_equal(out.cpu().numpy(), want)
    with pytest.raises(bs.BsError):
        bs.counts_noalloc(2048, e1, out)
