"""bs_counts_noalloc, the entry point for callers that cannot allocate device
memory (their memory belongs to a pre-allocated pool, or they must not touch
the CUDA allocator while they share the device).  Its counts must equal the
oracle's closed-triangle counts and those of bs_counts (the plan path)
exactly, on two calls in a row; the second call uses a different grid and
ring layout, so stale contents of the shared static scratch would show.  A
repeated call must leave the device's free memory unchanged (the first call
on a device loads the module that holds the array).  Wrongly typed or sized
tensors are refused by the binding before they reach the device.  Collected
last so that a failure here comes after every other test."""
import numpy as np
import pytest

import oracle
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


def _oracle_counts(nt, edges, ngrid=None):
    occ = None if ngrid is None else ngrid > 0
    T = oracle.counts(nt, edges, occupancy=occ)
    return np.array([T[i, j, l] for (i, j, l) in oracle.ring_triples(len(edges) - 1)])


def test_counts_noalloc_matches_oracle_and_plan_counts_twice():
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
    cases.append((40, synth.edges_linear(6, 20.0), ng))
    for nt, edges, ngh in cases:
        nb = len(edges) - 1
        ngrid = None if ngh is None else torch.from_numpy(ngh).cuda()
        out = torch.full((nb * (nb + 1) * (nb + 2) // 6,), -7, dtype=torch.int64, device="cuda")
        bs.counts_noalloc(nt, edges, out, ngrid=ngrid)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_array_equal(got, _oracle_counts(nt, edges, ngh))
        np.testing.assert_array_equal(got, _plan_counts(nt, edges, ngrid))
    # a repeated call reserves no device memory
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    bs.counts_noalloc(nt, edges, out, ngrid=ngrid)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    np.testing.assert_array_equal(out.cpu().numpy(), got)
    with pytest.raises(bs.BsError):
        bs.counts_noalloc(2048, e1, torch.zeros(1540, dtype=torch.int64, device="cuda"))


def test_counts_noalloc_refuses_wrong_tensors():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_10526_gb300 as bs
    edges = synth.edges_linear(4, 10.0)  # 4 rings: 20 ring triples
    with pytest.raises(ValueError):
        bs.counts_noalloc(32, edges, torch.zeros(20, dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        bs.counts_noalloc(32, edges, torch.zeros(19, dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):
        bs.counts_noalloc(32, edges, torch.zeros(20, dtype=torch.int64, device="cuda"),
                          ngrid=torch.ones((16, 16), dtype=torch.float32, device="cuda"))
