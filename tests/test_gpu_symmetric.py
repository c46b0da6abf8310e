"""Channel-symmetric accumulation (bs_mabs with accumulate = 2) against the
FP64 oracle and against the ordinary accumulation of the same cube.

A ring triple with a repeated ring is unchanged when the channels of the two
copies of that ring are exchanged (Eq. (estimator_t) multiplies the three
fields pointwise): (i, i, l) under nu1 <-> nu2, (i, j, j) under nu2 <-> nu3.
Over a cube block S x S x S the library contracts one ordering and fills in
the other before the collapse sums are read, so the folded plane, Eq. (dft)
and the exported sums must equal those of the ordinary accumulation of the
same cube.  The oracle's reference is the collapse of its full cube restricted
to S x S x S (tiny sizes) or its direct evaluation at sampled separations
(larger channel counts), including separations that only the fill-in
provides (d1 > d2 for (i, i, l), d2 > 0 for (i, j, j))."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {1: 1e-3, 2: 1e-4}


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _planes(plan, nc, torch):
    n2 = 2 * nc - 1
    dd = torch.empty((plan.batch, plan.ntrip, n2, n2), dtype=torch.float64, device="cuda")
    plan.mabs_delta(dd)
    b3 = torch.empty((plan.batch, plan.ntrip, nc, nc), dtype=torch.float64, device="cuda")
    plan.bs3d(b3)
    torch.cuda.synchronize()
    return dd.cpu().numpy(), b3.cpu().numpy()


def _kappa_err(got, want, babs):
    ok = ~np.isnan(want)
    assert np.array_equal(np.isnan(got), np.isnan(want)), "undefined bins differ"
    return np.max(np.abs(got[ok] - want[ok]) / babs[ok]) if ok.any() else 0.0


def _restricted(B, lo, hi):
    """The oracle's cube with every channel triple outside [lo, hi)^3 undefined."""
    R = np.array(B, dtype=np.float64, copy=True)
    keep = np.zeros(R.shape[1], bool)
    keep[lo:hi] = True
    m = keep[:, None, None] & keep[None, :, None] & keep[None, None, :]
    R[:, ~m] = np.nan
    return R


def _kinds(trips):
    return ["ii" if t[0] == t[1] else ("jj" if t[1] == t[2] else "-") for t in trips]


@pytest.mark.parametrize("precision,multires,flagged,S", [
    (1, True, False, (0, 16)), (1, False, True, (3, 14)), (2, True, True, (0, 16)),
    (2, False, False, (5, 16)), (1, True, True, (0, 9))])
def test_symmetric_cube_tiny_against_oracle(precision, multires, flagged, S):
    """64^2 grid, 16 channels, 8 linear rings (many repeated-ring triples):
    the folded plane of the symmetric cube against the oracle's collapse of
    the restricted cube, and plane + Eq. (dft) against the ordinary
    accumulation of the same cube."""
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt, nc = 64, 16
    edges = synth.edges_linear(8, 32)
    vis = synth.sky_visibilities(nt, nc, seed=1301)
    flags = synth.flag_mask_coarse_band(nc) if flagged else None
    lo, hi = S
    blk = (lo, hi) * 3
    plan = bs.Plan(nt, nc, edges, precision=precision, multires=multires)
    vd = torch.from_numpy(vis[None]).cuda()
    plan.grid_load(vd, chan_flags=flags)
    plan.mabs(block=blk, symmetric=True)
    d_sym, b_sym = _planes(plan, nc, torch)
    _, nnu_sym = plan.counts()
    plan.grid_load(vd, chan_flags=flags)  # resets the accumulators
    plan.mabs(block=blk, accumulate=True)
    d_ord, b_ord = _planes(plan, nc, torch)
    _, nnu_ord = plan.counts()
    plan.close()
    np.testing.assert_array_equal(nnu_sym, nnu_ord)
    ref = oracle.mabs_full(vis.astype(np.complex128), edges, chan_flags=flags)
    babs = oracle.mabs_full(np.abs(vis).astype(np.complex128), edges, chan_flags=flags)["B"].real
    bbar, cnt = oracle.collapse_fold(_restricted(ref["B"].real, lo, hi))
    bbar_abs, _ = oracle.collapse_fold(_restricted(babs, lo, hi))
    k0 = int(np.argmax(ref["T"] > 0))
    np.testing.assert_array_equal(nnu_sym, cnt[k0])
    tol = TOL[precision]
    e_sym = _kappa_err(d_sym[0], bbar, bbar_abs)
    e_ord = _kappa_err(d_ord[0], bbar, bbar_abs)
    kinds = _kinds(oracle.ring_triples(len(edges) - 1))
    print(f"precision {precision} multires {multires} flagged {flagged} S {S}: "
          f"kappa error symmetric {e_sym:.3e}, ordinary {e_ord:.3e}; "
          f"{kinds.count('ii')} (i,i,l) and {kinds.count('jj')} (i,j,j) triples")
    assert e_sym < tol, e_sym
    assert e_ord < tol, e_ord
    _check_dft(d_sym[0], b_sym[0], nc)
    _check_dft(d_ord[0], b_ord[0], nc)


def _check_dft(plane, b3, nc):
    """Eq. (dft) as bs_bs3d computed it (from the plan's sums) against the
    oracle's transform of the folded plane bs_mabs_delta returned: both read
    the filled-in sums, so they agree to the transform's FP32 rounding."""
    want = oracle.delay_dft(plane, nc).real
    for k in range(b3.shape[0]):
        m = np.abs(want[k]).max()
        if not np.isfinite(m) or m == 0:
            continue
        assert np.abs(b3[k] - want[k]).max() / m < 1e-5, k


def _sample_points(tri, trips, lo, hi, rng):
    """(i, j, l, d1, d2) on closable triples of each kind, with separations that
    the fill-in provides (d1 > d2 for (i, i, l), d2 > 0 for (i, j, j)), their
    computed counterparts, the axes and the origin."""
    w = hi - lo
    pts = []
    for kind in ("ii", "jj", "-"):
        ks = [k for k, t in enumerate(trips) if tri[k] > 0 and _kinds([t])[0] == kind]
        for k in ks[:: max(1, len(ks) // 3)][:3]:
            a = int(rng.integers(1, w - 1))
            b = int(rng.integers(-(w - 1 - a), a))  # a > b: nu1 > nu2 when i = j
            c = int(rng.integers(1, w - 1))
            for d in [(a, b), (b, a), (a - b, -b) if abs(a - b) < w else (a, 0),
                      (int(rng.integers(-(w - 1), w)), c), (0, 0), (w - 1, 0), (0, -(w - 1))]:
                pts.append((*trips[k], *d))
    return pts


@pytest.mark.parametrize("precision,nc,S,nb", [(1, 48, (0, 48), 4), (2, 40, (3, 37), 5),
                                               (1, 72, (8, 72), 4), (1, 168, (4, 164), 4)])
def test_symmetric_cube_sampled_against_oracle(precision, nc, S, nb):
    """Channel counts where some pair rectangles of a one-ring pair lie wholly
    below the diagonal (not contracted) and others straddle it, and a cube of
    160 channels (one launch per 128 x 128 sub-block of the pair plane): sampled
    separations of the folded plane against the oracle's direct evaluation
    over the cube, the whole plane against the ordinary accumulation, and the
    exported sums of the two equal."""
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt = 32
    edges = synth.edges_linear(nb, 15)
    vis = synth.sky_visibilities(nt, nc, seed=1400 + nc)
    lo, hi = S
    blk = (lo, hi) * 3
    plan = bs.Plan(nt, nc, edges, precision=precision, multires=True)
    vd = torch.from_numpy(vis[None]).cuda()
    plan.grid_load(vd)
    plan.mabs(block=blk, symmetric=True)
    d_sym, b_sym = _planes(plan, nc, torch)
    s_sym, nnu_sym = plan.delta_export()
    s_sym = s_sym.cpu().numpy()
    tri, _ = plan.counts()
    bound, _ = plan.error_bound()
    bound = bound.cpu().numpy()
    plan.grid_load(vd)
    plan.mabs(block=blk, accumulate=True)
    d_ord, _ = _planes(plan, nc, torch)
    s_ord, nnu_ord = plan.delta_export()
    s_ord = s_ord.cpu().numpy()
    plan.close()
    np.testing.assert_array_equal(nnu_sym, nnu_ord)
    trips = oracle.ring_triples(nb)
    pts = _sample_points(tri, trips, lo, hi, np.random.default_rng(nc))
    want, cnt = oracle.delta_points(vis.astype(np.complex128), edges, pts, nu_lo=lo, nu_hi=hi)
    babs, _ = oracle.delta_points(np.abs(vis).astype(np.complex128), edges, pts, nu_lo=lo,
                                  nu_hi=hi)
    n1 = nc - 1
    idx = [trips.index(tuple(p[:3])) for p in pts]
    got = np.array([d_sym[0, k, p[3] + n1, p[4] + n1] for k, p in zip(idx, pts)])
    ok = cnt > 0
    assert ok.sum() >= len(pts) // 2
    assert np.array_equal(np.isnan(got), ~ok)
    err = np.abs(got[ok] - want.real[ok])
    ek = err / babs.real[ok]
    print(f"precision {precision} nc {nc} S {S}: {ok.sum()} sampled points, "
          f"kappa error max {ek.max():.3e}")
    assert ek.max() < TOL[precision], ek
    beta = np.array([bound[0, k] for k in idx])[ok]
    assert np.all(err <= beta + 1e-13 * babs.real[ok])
    # whole planes: both within the error bound of the exact value; raw sums:
    # the same entries filled
    both = ~np.isnan(d_ord)
    assert np.array_equal(both, ~np.isnan(d_sym))
    for k in np.flatnonzero(tri > 0):
        diff = np.abs(d_sym[0, k] - d_ord[0, k])[both[0, k]]
        assert np.all(diff <= 2 * bound[0, k] * (1 + 1e-9)), k
    assert np.array_equal(s_sym == 0, s_ord == 0)
    _check_dft(d_sym[0], b_sym[0], nc)


def test_symmetric_accumulation_rules():
    """Refusals (FP32 plan, a block that is not a cube, a full-cube output, a
    symmetric cube after ordinary blocks) and the allowed sequences: ordinary
    blocks after symmetric cubes, two symmetric cubes, and import after a
    symmetric cube, each equal to the ordinary accumulation of the same
    channel triples."""
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt, nc = 32, 24
    edges = synth.edges_linear(4, 15)
    vis = synth.sky_visibilities(nt, nc, seed=1500)
    vd = torch.from_numpy(vis[None]).cuda()

    fp = bs.Plan(nt, nc, edges, precision=0)
    fp.grid_load(vd)
    with pytest.raises(bs.BsError) as e:
        fp.mabs(block=(0, 8) * 3, symmetric=True)
    assert e.value.status == 8  # BS_ERR_UNSUPPORTED
    fp.close()

    plan = bs.Plan(nt, nc, edges, precision=1, multires=True)
    plan.grid_load(vd)
    with pytest.raises(bs.BsError) as e:
        plan.mabs(block=(0, 8, 0, 8, 0, 12), symmetric=True)
    assert e.value.status == 1  # BS_ERR_ARG
    full = torch.zeros((1, plan.ntrip, nc, nc, nc), dtype=torch.float64, device="cuda")
    with pytest.raises(bs.BsError) as e:
        plan.mabs(block=(0, 8) * 3, out_full=full, symmetric=True)
    assert e.value.status == 1
    plan.mabs(block=(0, 8, 8, 16, 0, 24), accumulate=True)
    with pytest.raises(bs.BsError) as e:
        plan.mabs(block=(0, 8) * 3, symmetric=True)
    assert e.value.status == 7  # BS_ERR_STATE

    # reference: ordinary accumulation of two cubes and one block
    cubes = [(0, 12) * 3, (12, 24) * 3]
    extra = (0, 12, 12, 24, 0, 24)
    plan.grid_load(vd)
    for c in cubes:
        plan.mabs(block=c, accumulate=True)
    plan.mabs(block=extra, accumulate=True)
    d_ref, _ = _planes(plan, nc, torch)
    bound, _ = plan.error_bound()
    bound = bound.cpu().numpy()
    tri, nnu_ref = plan.counts()

    def close_to_ref(d):
        ok = ~np.isnan(d_ref)
        assert np.array_equal(ok, ~np.isnan(d))
        for k in np.flatnonzero(tri > 0):
            diff = np.abs(d[0, k] - d_ref[0, k])[ok[0, k]]
            assert np.all(diff <= 2 * bound[0, k] * (1 + 1e-9)), k

    # symmetric cubes, a read in between, then an ordinary block
    plan.grid_load(vd)
    plan.mabs(block=cubes[0], symmetric=True)
    _planes(plan, nc, torch)  # fills in; accumulation continues afterwards
    plan.mabs(block=cubes[1], symmetric=True)
    plan.mabs(block=extra, accumulate=True)
    d, _ = _planes(plan, nc, torch)
    assert np.array_equal(plan.counts()[1], nnu_ref)
    close_to_ref(d)

    # export of symmetric cubes, imported and added to an ordinary block
    plan.grid_load(vd)
    plan.mabs(block=cubes[0], symmetric=True)
    plan.mabs(block=cubes[1], symmetric=True)
    sums, nnu = plan.delta_export()
    plan.grid_load(vd)
    plan.mabs(block=extra, accumulate=True)
    plan.delta_import(sums, nnu, add=True)
    with pytest.raises(bs.BsError) as e:  # imported sums count as ordinary ones
        plan.mabs(block=cubes[0], symmetric=True)
    assert e.value.status == 7
    d, _ = _planes(plan, nc, torch)
    close_to_ref(d)
    plan.close()
