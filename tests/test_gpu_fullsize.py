"""Parity at the full MWA-like size: 256^2 grid, 768 channels, 20 log rings
(M = 384), one 64^3 channel block per bs_mabs call, and the exact
128 x 128 x 256 block the benchmark times.  The full channel cube cannot be
stored, so the check samples the folded collapsed plane: for chosen ring
triples and separations the oracle evaluates the mean of Eq. (estimator_t)
over the block's channel triples directly (closed-triangle enumeration), and
the kappa-normalised error is formed with the oracle's value on |V|.  At
every sampled point the error bound of bs_mabs_error_bound must cover the
error, and well-conditioned points (kappa u <= tol / 10) must meet the
tolerance in relative error.  Counts of all 1540 ring triples are compared
exactly.  The benchmark's channel-symmetric 256^3 cube is sampled the same
way.  A 512^2 grid with 24 log rings (image side 768) is sampled on a small
channel block."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

NT, NC, NB = 256, 768, 20
EDGES = synth.edges_log(NB, 4.41, 128.0)
BLOCK = 64
UNIT = {0: 2.0 ** -24, 1: 2.0 ** -17, 2: 2.0 ** -22}


def _check_points(got, want, babs, beta, precision, tol, label):
    """kappa-normalised error, bound coverage and the relative error of
    well-conditioned points at sampled points."""
    err = np.abs(got - want.real)
    ek = err / babs.real
    kappa = babs.real / np.abs(want.real)
    good = kappa * UNIT[precision] <= tol / 10
    print(f"{label}: kappa-normalised error max {ek.max():.3e}; error/bound max "
          f"{(err / beta).max():.2e}; kappa range {kappa.min():.3g}..{kappa.max():.3g}, "
          f"{good.sum()} of {good.size} well-conditioned")
    assert ek.max() < tol, ek
    assert np.all(err <= beta + 1e-13 * babs.real), err / beta
    assert np.all(err[good] / np.abs(want.real[good]) <= tol)


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
    bound, _ = plan.error_bound()
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
    beta = np.array([bound[0, trips.index(tuple(p[:3]))].item() for p in pts])
    plan.close()
    assert np.all(cnt > 0)
    _check_points(got, want, babs, beta, precision, tol,
                  f"precision {precision} multires {multires}")


def test_bench_block_sampled_parity():
    """The benchmark's exact launch: split BF16, per-triple image sides, the
    128 x 128 x 256 channel block (nu3 over 256 channels)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_10526_gb300 as bs
    vis = synth.sky_visibilities(NT, NC, 2000, f_ng=0.5, sigma=0.5)
    plan = bs.Plan(NT, NC, EDGES, precision=1, multires=True)
    plan.grid_load(torch.from_numpy(vis[None]).cuda())
    blk = (0, 128, 0, 128, 0, 256)
    plan.mabs(block=blk, accumulate=True)
    n2 = 2 * NC - 1
    out = torch.empty((1, plan.ntrip, n2, n2), dtype=torch.float64, device="cuda")
    plan.mabs_delta(out)
    bound, _ = plan.error_bound()
    tri, _ = plan.counts()
    torch.cuda.synchronize()
    trips = oracle.ring_triples(NB)
    idx = [k for k in range(len(trips)) if tri[k] > 0]
    chosen = idx[:4] + [idx[len(idx) // 4], idx[len(idx) // 3]]
    ds = [(0, 0), (100, -3), (-17, 90), (127, 127), (-200, -90), (-250, -130)]  # all sampled
    pts = [(*trips[k], *ds[n % len(ds)]) for n, k in enumerate(chosen)]
    pts += [(*trips[k], 1, 0) for k in chosen[:3]]
    sub = vis[:256].astype(np.complex128)
    want, cnt = oracle.delta_points(sub, EDGES, pts, block=blk)
    babs, _ = oracle.delta_points(np.abs(sub), EDGES, pts, block=blk)
    got = np.array([out[0, trips.index(tuple(p[:3])), p[3] + NC - 1, p[4] + NC - 1].item()
                    for p in pts])
    beta = np.array([bound[0, trips.index(tuple(p[:3]))].item() for p in pts])
    plan.close()
    assert np.all(cnt > 0)
    _check_points(got, want, babs, beta, 1, 1e-3, "bench block 128 x 128 x 256")


def test_bench_symmetric_cube_sampled_parity():
    """The benchmark's exact launch: split BF16, per-triple image sides, the
    256^3 channel cube with the channel symmetry of repeated rings
    (accumulate = 2).  Points on (i, i, l) and (i, j, j) triples at
    separations that the contraction computes and ones that only the fill-in
    provides, and on triples of three different rings."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_10526_gb300 as bs
    vis = synth.sky_visibilities(NT, NC, 2000, f_ng=0.5, sigma=0.5)
    plan = bs.Plan(NT, NC, EDGES, precision=1, multires=True)
    plan.grid_load(torch.from_numpy(vis[None]).cuda())
    w = 256
    plan.mabs(block=(0, w) * 3, symmetric=True)
    n2 = 2 * NC - 1
    out = torch.empty((1, plan.ntrip, n2, n2), dtype=torch.float64, device="cuda")
    plan.mabs_delta(out)
    bound, _ = plan.error_bound()
    tri, _ = plan.counts()
    torch.cuda.synchronize()
    trips = oracle.ring_triples(NB)
    pts = []
    for kind in ("ii", "jj", "-"):
        ks = [k for k, t in enumerate(trips) if tri[k] > 0 and
              kind == ("ii" if t[0] == t[1] else ("jj" if t[1] == t[2] else "-"))]
        for n, k in enumerate(ks[:2] + [ks[len(ks) // 3]]):
            # (d1 > d2) is filled in for (i, i, l), (d2 > 0) for (i, j, j)
            ds = [(120, -30), (-30, 120), (150, 30), (-100, -200), (0, 0), (255 - n, 1)]
            for d in ds[:2] if n == 2 else ds:  # fewer points on the larger rings
                pts.append((*trips[k], *d))
    sub = vis[:w].astype(np.complex128)
    want, cnt = oracle.delta_points(sub, EDGES, pts)
    babs, _ = oracle.delta_points(np.abs(sub), EDGES, pts)
    got = np.array([out[0, trips.index(tuple(p[:3])), p[3] + NC - 1, p[4] + NC - 1].item()
                    for p in pts])
    beta = np.array([bound[0, trips.index(tuple(p[:3]))].item() for p in pts])
    plan.close()
    assert np.all(cnt > 0)
    _check_points(got, want, babs, beta, 1, 1e-3, "bench cube 256^3, channel-symmetric")


@pytest.mark.parametrize("precision,multires", [(1, True), (0, False)])
def test_grid_512_with_24_log_rings(precision, multires):
    """512^2 grid, 24 log rings |U| in [4.41, 256): a single image side of 768
    (FP32), or per-triple sides up to 768 (split BF16); 8 channels.  Points
    on ring triples at the largest side and at small ones."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_10526_gb300 as bs
    nt, nc, nb = 512, 8, 24
    edges = synth.edges_log(nb, 4.41, 256.0)
    vis = synth.sky_visibilities(nt, nc, 4000, f_ng=0.5, sigma=0.5)
    plan = bs.Plan(nt, nc, edges, precision=precision, multires=multires)
    plan.grid_load(torch.from_numpy(vis[None]).cuda())
    plan.mabs(accumulate=True)
    n2 = 2 * nc - 1
    out = torch.empty((1, plan.ntrip, n2, n2), dtype=torch.float64, device="cuda")
    plan.mabs_delta(out)
    bound, _ = plan.error_bound()
    tri, _ = plan.counts()
    sides = plan.trip_sides()
    torch.cuda.synchronize()
    assert plan.M == 768 and sides.max() == 768
    trips = oracle.ring_triples(nb)
    Tor = oracle.counts(nt, edges)
    np.testing.assert_array_equal(tri, [Tor[t] for t in trips])
    big = [k for k in range(len(trips)) if tri[k] > 0 and sides[k] == 768 and trips[k][0] <= 12]
    small = [k for k in range(len(trips)) if tri[k] > 0 and trips[k][2] <= 6]
    chosen = big[:3] + small[:3]
    assert len(chosen) == 6
    pts = [(*trips[k], d1, d2) for k in chosen for d1, d2 in ((0, 0), (3, -2))]
    want, cnt = oracle.delta_points(vis.astype(np.complex128), edges, pts)
    babs, _ = oracle.delta_points(np.abs(vis).astype(np.complex128), edges, pts)
    got = np.array([out[0, trips.index(tuple(p[:3])), p[3] + nc - 1, p[4] + nc - 1].item()
                    for p in pts])
    beta = np.array([bound[0, trips.index(tuple(p[:3]))].item() for p in pts])
    plan.close()
    assert np.all(cnt > 0)
    tol = {0: 1e-5, 1: 1e-3}[precision]
    _check_points(got, want, babs, beta, precision, tol, f"512^2 precision {precision}")


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
