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
                                                    (0, False, 1e-5)])
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
