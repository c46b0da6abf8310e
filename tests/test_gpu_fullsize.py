"""Parity at the full MWA-like size, in the launch configuration bench.py
times: 256^2 grid, 768 channels, 20 log rings (M = 384), one 64^3 channel
block per bs_mabs call.  The full channel cube cannot be stored, so the
check samples the folded collapsed plane: for chosen ring triples and
separations the oracle evaluates the mean of Eq. (estimator_t) over the
block's channel triples directly (closed-triangle enumeration), and the
kappa-normalised error is formed with the oracle's value on |V|.  Counts of
all 1540 ring triples are compared exactly."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

NT, NC, NB = 256, 768, 20
EDGES = synth.edges_log(NB, 4.41, 128.0)
BLOCK = 64


def _points(T, trips):
    """Sample (i, j, l, d1, d2): closable triples spread over the ring sizes,
    separations inside the block (origin, axes, diagonal, ragged)."""
    idx = [k for k, t in enumerate(trips) if T[k] > 0]
    # small rings are cheap for the oracle; include some large ones too
    chosen = idx[:6] + [idx[len(idx) // 3], idx[len(idx) // 2], idx[-40], idx[-1]]
    ds = [(0, 0), (5, -3), (-17, 2), (31, 31), (-40, 20), (12, -50)]  # spread < 64
    pts = []
    for n, k in enumerate(chosen):
        d1, d2 = ds[n % len(ds)]
        pts.append((*trips[k], d1, d2))
        pts.append((*trips[k], 1, 0))
    return pts, chosen


@pytest.mark.parametrize("precision,multires,tol", [(1, True, 1e-3), (1, False, 1e-3),
                                                    (2, True, 1e-4), (0, False, 1e-5)])
def test_mwa_block_sampled_parity(precision, multires, tol):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_10526_gb300 as bs
    vis = synth.sky_visibilities(NT, NC, 2000, f_ng=0.5, sigma=0.5)
    plan = bs.Plan(NT, NC, EDGES, precision=precision, multires=multires)
    assert plan.M == 384
    plan.grid_load(torch.from_numpy(vis[None]).cuda())
    blk = (0, BLOCK, 0, BLOCK, 0, BLOCK)
    plan.mabs(block=blk, accumulate=True)
    n2 = 2 * NC - 1
    out = torch.empty((1, plan.ntrip, n2, n2), dtype=torch.float64, device="cuda")
    plan.mabs_delta(out)
    tri, _ = plan.counts()
    torch.cuda.synchronize()
    Tor = oracle.counts(NT, EDGES)
    trips = oracle.ring_triples(NB)
    np.testing.assert_array_equal(tri, [Tor[t] for t in trips])
    pts, _ = _points(tri, trips)
    sub = vis[:BLOCK].astype(np.complex128)
    want, cnt = oracle.delta_points(sub, EDGES, pts)
    babs, _ = oracle.delta_points(np.abs(sub), EDGES, pts)
    got = np.array([out[0, trips.index(tuple(p[:3])), p[3] + NC - 1, p[4] + NC - 1].item()
                    for p in pts])
    plan.close()
    assert np.all(cnt > 0)
    err = np.abs(got - want.real) / babs.real
    print(f"precision {precision} multires {multires}: sampled kappa-normalised error max "
          f"{err.max():.3e}")
    assert err.max() < tol, err


def test_mwa_delay_transform_full_size():
    """Eq. (dft) at the full size (768 channels, multi-row delay-transform
    passes): the GPU's 3D bispectrum of sampled ring triples against the
    oracle's literal double sum applied to the GPU's own folded plane (the
    plane itself is checked against the oracle above).  FP32 FFTs of length
    768 against an FP64 DFT: 1e-4 of the largest |B| of each triple."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_10526_gb300 as bs
    vis = synth.sky_visibilities(NT, NC, 2001, f_ng=0.5, sigma=0.5)
    plan = bs.Plan(NT, NC, EDGES, precision=1, multires=True)
    plan.grid_load(torch.from_numpy(vis[None]).cuda())
    plan.mabs(block=(0, 128, 0, 128, 0, 256), accumulate=True)
    n2 = 2 * NC - 1
    dd = torch.empty((1, plan.ntrip, n2, n2), dtype=torch.float64, device="cuda")
    b3 = torch.empty((1, plan.ntrip, NC, NC), dtype=torch.float64, device="cuda")
    plan.mabs_delta(dd)
    plan.bs3d(b3)
    tri, _ = plan.counts()
    torch.cuda.synchronize()
    closable = np.flatnonzero(tri > 0)
    sample = closable[np.linspace(0, closable.size - 1, 5).astype(int)]
    for k in sample:
        plane = dd[0, k].cpu().numpy()
        want = oracle.delay_dft(plane, NC).real
        got = b3[0, k].cpu().numpy()
        err = np.abs(got - want).max() / np.abs(want).max()
        print(f"ring triple {k}: max |B3_gpu - B3_oracle| / max|B3| = {err:.2e}")
        assert err < 1e-4, (k, err)
    # ring triples without closed triangles are zero
    zero = torch.from_numpy(np.flatnonzero(tri == 0)).cuda()
    assert float(b3[0].index_select(0, zero).abs().max()) == 0.0
    plan.close()
