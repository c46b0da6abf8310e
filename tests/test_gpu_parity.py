"""GPU parity: libbs (through its C ABI) against the FP64 oracle on the same
seeded inputs.

Error measure (per estimator bin): the oracle evaluates Eq. (estimator_t)
twice, on V and on |V|; the second gives B_abs = (1/A) sum_t |X1 X2 X3| / T,
the size of the terms that cancel in the bin.  The kappa-normalised error
e = |B_gpu - B_fp64| / B_abs must stay below 1e-5 for the FP32 path (the
FP32 target; the FFTs and the contraction round at ~6e-8 relative to the
terms, times the log2 M FFT stages and the growth of long FP32 sums).
Counts are integers and must be bit-exact; undefined bins must coincide."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5
# split-BF16 tensor-core path: operands carry 16 significant bits (hi + lo),
# products lose ~2^-16 relative; target 1e-3 kappa-normalised
TOL_SPLIT = 1e-3
# split-FP16 path (precision 2): the same three products on FP16 hi + lo parts
# of power-of-two-scaled operands, 22 significant bits (~3 x 2^-22 per term):
# held to 1e-4, ten times tighter than split BF16
TOL = {0: TOL_FP32, 1: TOL_SPLIT, 2: 1e-4}
SPLIT_CASES = [(1, False), (1, True), (2, False), (2, True)]


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _run(vis, edges, flags=None, ngrid=None, precision=0, block=None, full=True, batch_vis=None,
         norm_A=1.0, r=1.0, rprime=1.0, dnu_c=1.0, multires=False):
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    v = vis if batch_vis is None else batch_vis
    if v.ndim == 3:
        v = v[None]
    batch, nc, nt, _ = v.shape
    plan = bs.Plan(nt, nc, edges, precision=precision, batch=batch, norm_A=norm_A, r=r,
                   rprime=rprime, dnu_c=dnu_c, multires=multires)
    vd = torch.from_numpy(np.ascontiguousarray(v.astype(np.complex64))).cuda()
    gd = None if ngrid is None else torch.from_numpy(ngrid.astype(np.float32)).cuda()
    plan.grid_load(vd, ngrid=gd, chan_flags=flags)
    out = {}
    fd = None
    if full:
        fd = torch.full((batch, plan.ntrip, nc, nc, nc), 12345.0, dtype=torch.float64,
                        device="cuda")
    plan.mabs(block=block, out_full=fd, accumulate=True)
    dd = torch.empty((batch, plan.ntrip, 2 * nc - 1, 2 * nc - 1), dtype=torch.float64,
                     device="cuda")
    plan.mabs_delta(dd)
    bd = torch.empty((batch, plan.ntrip, nc, nc), dtype=torch.float64, device="cuda")
    plan.bs3d(bd)
    torch.cuda.synchronize()
    out["full"] = None if fd is None else fd.cpu().numpy()
    out["delta"] = dd.cpu().numpy()
    out["bs3d"] = bd.cpu().numpy()
    out["T"], out["nnu"] = plan.counts()
    out["M"] = plan.M
    plan.close()
    return out


def _kappa_err(got, want, babs):
    ok = ~np.isnan(want)
    assert np.array_equal(np.isnan(got), np.isnan(want)), "undefined bins differ"
    return np.max(np.abs(got[ok] - want[ok]) / babs[ok]) if ok.any() else 0.0


def _oracle(vis, edges, flags=None, ngrid=None, norm_A=1.0):
    ref = oracle.mabs_full(vis.astype(np.complex128), edges, chan_flags=flags, ngrid=ngrid,
                           norm_A=norm_A)
    babs = oracle.mabs_full(np.abs(vis).astype(np.complex128), edges, chan_flags=flags,
                            ngrid=ngrid, norm_A=norm_A)["B"].real
    return ref, babs


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_three_mode_golden_gpu(precision):
    nt = 8
    vis = np.zeros((1, nt, nt), np.complex64)
    for (u, v), z in (((1, 0), 1 + 2j), ((1, 1), 0.5 - 1j), ((-2, -1), -1 + 0.25j)):
        vis[0, v + nt // 2, u + nt // 2] = z
        vis[0, -v + nt // 2, -u + nt // 2] = np.conj(z)
    out = _run(vis, [1, 2, 3, 4], precision=precision)
    assert out["T"][0] == 24 and out["T"][1] == 32  # (0,0,0), (0,0,1): hand counts
    assert out["full"][0, 1, 0, 0, 0] == pytest.approx(-0.3125, abs=1e-6 if precision == 0 else 1e-4)
    assert abs(out["full"][0, 0, 0, 0, 0]) < 1e-6


@pytest.mark.parametrize("precision,multires", [(0, False), (0, True)] + SPLIT_CASES)
@pytest.mark.parametrize("flagged", [False, True])
def test_tiny_config_full_cube(flagged, precision, multires):
    """64^2 grid, 16 channels, 8 linear rings (and the coarse-band flags):
    every ring triple x channel triple against the oracle, FP32 SIMT and
    split-BF16 tensor-core contraction."""
    nt, nc = 64, 16
    edges = synth.edges_linear(8, 32)
    vis = synth.sky_visibilities(nt, nc, seed=1001)
    flags = synth.flag_mask_coarse_band(nc) if flagged else None
    out = _run(vis, edges, flags=flags, precision=precision, multires=multires)
    ref, babs = _oracle(vis, edges, flags)
    np.testing.assert_array_equal(out["T"], ref["T"])
    e = _kappa_err(out["full"][0], ref["B"].real, babs)
    print(f"precision {precision} multires {multires} flagged {flagged}: "
          f"max kappa-normalised error {e:.3e}")
    tol = TOL[precision]
    assert e < tol, e
    bbar, cnt = oracle.collapse_fold(ref["B"].real)
    bbar_abs, _ = oracle.collapse_fold(babs)
    k0 = int(np.argmax(ref["T"] > 0))
    np.testing.assert_array_equal(out["nnu"], cnt[k0])
    e = _kappa_err(out["delta"][0], bbar, bbar_abs)
    assert e < tol, e
    b3 = oracle.delay_dft(bbar, nc).real
    b3_scale = np.abs(oracle.delay_dft(bbar_abs, nc)).max(axis=(-1, -2), keepdims=True)
    keep = ref["T"] > 0
    err3 = np.abs(out["bs3d"][0][keep] - b3[keep]) / b3_scale[keep]
    assert err3.max() < tol, err3.max()


@pytest.mark.parametrize("precision,multires", [(0, False), (0, True)] + SPLIT_CASES)
def test_ragged_sizes_occupancy_and_blocks(precision, multires):
    """Non-tile-multiple sizes: nt = 40, 11 channels (non-smooth: direct DFT in
    the delay transform), log rings, empty cells with N_g in {0, 1, 2, 3},
    one flagged channel, and three channel blocks that tile the cube."""
    nt, nc = 40, 11
    edges = synth.edges_log(5, 1.5, 19.0)
    vis = synth.sky_visibilities(nt, nc, seed=42)
    r = synth.rng(43)
    ngrid = r.integers(0, 4, size=(nt, nt)).astype(np.float32)
    # same sampling at U and -U: cell (iv, iu) pairs with (nt - iv, nt - iu)
    ngrid[1:, 1:] = np.maximum(ngrid[1:, 1:], ngrid[1:, 1:][::-1, ::-1])
    flags = np.zeros(nc, np.uint8)
    flags[4] = 1
    ref, babs = _oracle(vis, edges, flags, ngrid=ngrid)
    occ = oracle.ring_labels(nt, edges, occupancy=ngrid > 0)
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    plan = bs.Plan(nt, nc, edges, precision=precision, multires=multires)
    plan.grid_load(torch.from_numpy(vis[None]).cuda(), ngrid=torch.from_numpy(ngrid).cuda(),
                   chan_flags=flags)
    full = torch.full((1, plan.ntrip, nc, nc, nc), np.nan, dtype=torch.float64, device="cuda")
    for blk in [(0, 5, 0, 11, 0, 11), (5, 11, 0, 7, 0, 11), (5, 11, 7, 11, 0, 11)]:
        plan.mabs(block=blk, out_full=full, accumulate=True)
    dd = torch.empty((1, plan.ntrip, 2 * nc - 1, 2 * nc - 1), dtype=torch.float64, device="cuda")
    plan.mabs_delta(dd)
    bd = torch.empty((1, plan.ntrip, nc, nc), dtype=torch.float64, device="cuda")
    plan.bs3d(bd)
    tri, nnu = plan.counts()
    torch.cuda.synchronize()
    Tocc = oracle.counts(nt, edges, occupancy=ngrid > 0)
    trips = oracle.ring_triples(len(edges) - 1)
    np.testing.assert_array_equal(tri, [Tocc[t] for t in trips])
    assert occ is not None
    tol = TOL[precision]
    e = _kappa_err(full[0].cpu().numpy(), ref["B"].real, babs)
    assert e < tol, e
    bbar, cnt = oracle.collapse_fold(ref["B"].real)
    bbar_abs, _ = oracle.collapse_fold(babs)
    np.testing.assert_array_equal(nnu, cnt[int(np.argmax(ref["T"] > 0))])
    e = _kappa_err(dd[0].cpu().numpy(), bbar, bbar_abs)
    assert e < tol, e
    b3 = oracle.delay_dft(bbar, nc).real
    b3_scale = np.abs(oracle.delay_dft(bbar_abs, nc)).max(axis=(-1, -2), keepdims=True)
    keep = ref["T"] > 0
    err3 = np.abs(bd[0].cpu().numpy()[keep] - b3[keep]) / b3_scale[keep]
    assert err3.max() < tol, err3.max()
    plan.close()


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_batch_and_scales(precision):
    """Two realisations in one plan; A, r, r', dnu_c scale factors."""
    nt, nc = 32, 8
    edges = synth.edges_linear(4, 16)
    v = np.stack([synth.sky_visibilities(nt, nc, seed=s) for s in (3, 4)])
    A, r, rp, dnu = 2.0, 1.5, 0.8, 0.25
    out = _run(None, edges, batch_vis=v, norm_A=A, r=r, rprime=rp, dnu_c=dnu, precision=precision)
    tol = TOL[precision]
    for b in range(2):
        ref, babs = _oracle(v[b], edges, norm_A=A)
        e = _kappa_err(out["full"][b], ref["B"].real, babs)
        assert e < tol, (b, e)
        bbar, _ = oracle.collapse_fold(ref["B"].real)
        b3 = oracle.delay_dft(bbar, nc, r, rp, dnu).real
        b3_scale = np.abs(oracle.delay_dft(oracle.collapse_fold(babs)[0], nc, r, rp, dnu)).max()
        keep = ref["T"] > 0
        assert np.abs(out["bs3d"][b][keep] - b3[keep]).max() / b3_scale < tol


@pytest.mark.parametrize("precision,multires", [(0, False), (0, True)] + SPLIT_CASES)
def test_degenerate_cases(precision, multires):
    """One channel (the single-frequency ABS special case), a single ring,
    an empty ring, every channel flagged, and the constant field (B = 1/A)."""
    nt = 16
    tol = TOL[precision]
    vis = synth.sky_visibilities(nt, 1, seed=9)
    edges = [1.0, 3.0, 3.1, 7.0]  # ring 1 holds no cell
    out = _run(vis, edges, precision=precision, multires=multires)
    ref, babs = _oracle(vis, edges)
    assert _kappa_err(out["full"][0], ref["B"].real, babs) < tol
    out = _run(vis, [1.0, 7.0], precision=precision, multires=multires)
    ref, babs = _oracle(vis, [1.0, 7.0])
    assert _kappa_err(out["full"][0], ref["B"].real, babs) < tol
    vis4 = synth.sky_visibilities(nt, 4, seed=10)
    out = _run(vis4, [1.0, 4.0, 7.0], flags=np.ones(4, np.uint8), precision=precision, multires=multires)
    assert np.all(np.isnan(out["full"])) and np.all(np.isnan(out["delta"]))
    assert np.all(out["bs3d"] == 0)
    ones = np.ones((3, nt, nt), np.complex64)
    out = _run(ones, [1.0, 4.0, 7.0], norm_A=4.0, precision=precision, multires=multires)
    f = out["full"][0]
    ok = ~np.isnan(f)
    np.testing.assert_allclose(f[ok], 0.25, rtol=1e-5 if precision == 0 else 1e-3)


@pytest.mark.parametrize("amp", [1e-15, 1e15])
def test_split_fp16_amplitude_range(amp):
    """Split FP16 keeps FP16 operands in range by power-of-two field scales
    chosen from each field's largest value: visibilities scaled by 1e-15 or
    1e15 give B scaled by amp^3 at the same kappa-normalised error (two
    realisations 3e3 apart in amplitude share one plan).  Log rings on a 48^2
    grid with few closed triangles per bin: split BF16 measures 1e-4 to 2.4e-4
    here and overflows FP32 at 1e15."""
    nt, nc = 48, 12
    edges = synth.edges_log(6, 1.5, 23.0)
    v = np.stack([synth.sky_visibilities(nt, nc, seed=s) for s in (21, 22)])
    v[1] *= 3.0e3
    ref = [_oracle(v[b], edges) for b in range(2)]
    out = _run(None, edges, batch_vis=(v * amp).astype(np.complex64), precision=2, multires=True)
    for b in range(2):
        e = _kappa_err(out["full"][b] / amp ** 3, ref[b][0]["B"].real, ref[b][1])
        print(f"amp {amp:g} realisation {b}: max kappa-normalised error {e:.3e}")
        assert e < TOL[2], (b, e)


@pytest.mark.parametrize("precision,multires", [(1, True), (0, False)])
def test_closable_layouts_match_full(precision, multires):
    """bs_mabs_delta_closable / bs_bs3d_closable hold exactly the planes of the
    full layouts whose ring triple has closed triangles, in ascending order,
    bit for bit; two realisations, one flagged channel."""
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt, nc = 40, 11
    edges = synth.edges_log(5, 1.5, 19.0)
    v = np.stack([synth.sky_visibilities(nt, nc, seed=s) for s in (61, 62)])
    flags = np.zeros(nc, np.uint8)
    flags[3] = 1
    plan = bs.Plan(nt, nc, edges, precision=precision, batch=2, multires=multires)
    plan.grid_load(torch.from_numpy(v).cuda(), chan_flags=flags)
    plan.mabs(accumulate=True)
    tri, _ = plan.counts()
    clos = np.flatnonzero(tri > 0)
    assert plan.n_closable == clos.size and 0 < clos.size < plan.ntrip
    n2 = 2 * nc - 1
    dd = torch.empty((2, plan.ntrip, n2, n2), dtype=torch.float64, device="cuda")
    dc = torch.full((2, clos.size, n2, n2), 7.0, dtype=torch.float64, device="cuda")
    bd = torch.empty((2, plan.ntrip, nc, nc), dtype=torch.float64, device="cuda")
    bc = torch.full((2, clos.size, nc, nc), 7.0, dtype=torch.float64, device="cuda")
    plan.mabs_delta(dd)
    plan.mabs_delta_closable(dc)
    plan.bs3d(bd)
    plan.bs3d_closable(bc)
    torch.cuda.synchronize()
    idx = torch.from_numpy(clos).cuda()
    np.testing.assert_array_equal(dc.cpu().numpy(), dd.index_select(1, idx).cpu().numpy())
    np.testing.assert_array_equal(bc.cpu().numpy(), bd.index_select(1, idx).cpu().numpy())
    plan.close()


@pytest.mark.parametrize("precision,multires", [(1, True), (0, False)])
def test_reload_resets_the_accumulators(precision, multires):
    """A grid load resets the collapse sums by zeroing only the separations
    the previous blocks touched: load, accumulate block A, reload with other
    visibilities, accumulate block B; the collapse and the delay transform
    equal those of a fresh plan that only saw the second load and block B."""
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt, nc = 40, 12
    edges = synth.edges_log(5, 1.5, 19.0)
    v1 = torch.from_numpy(synth.sky_visibilities(nt, nc, seed=91)[None]).cuda()
    v2 = torch.from_numpy(synth.sky_visibilities(nt, nc, seed=92)[None]).cuda()
    blk_a, blk_b = (0, 6, 0, 12, 0, 12), (6, 12, 0, 5, 4, 12)

    def outputs(plan):
        n2 = 2 * nc - 1
        dd = torch.empty((1, plan.ntrip, n2, n2), dtype=torch.float64, device="cuda")
        bd = torch.empty((1, plan.ntrip, nc, nc), dtype=torch.float64, device="cuda")
        plan.mabs_delta(dd)
        plan.bs3d(bd)
        torch.cuda.synchronize()
        return dd.cpu().numpy(), bd.cpu().numpy()

    p = bs.Plan(nt, nc, edges, precision=precision, multires=multires)
    p.grid_load(v1)
    p.mabs(block=blk_a, accumulate=True)
    outputs(p)
    p.grid_load(v2)
    p.mabs(block=blk_b, accumulate=True)
    got = outputs(p)
    q = bs.Plan(nt, nc, edges, precision=precision, multires=multires)
    q.grid_load(v2)
    q.mabs(block=blk_b, accumulate=True)
    want = outputs(q)
    for g, w in zip(got, want):
        assert np.array_equal(np.isnan(g), np.isnan(w))
        ok = ~np.isnan(w)
        assert np.abs(g[ok] - w[ok]).max() <= 1e-9 * max(np.abs(w[ok]).max(), 1e-300)
    p.close()
    q.close()


def test_hermitian_check():
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt, nc = 16, 2
    vis = synth.sky_visibilities(nt, nc, seed=1)
    plan = bs.Plan(nt, nc, [1.0, 4.0, 7.0])
    v = torch.from_numpy(vis[None]).cuda()
    assert plan.check_hermitian(v, 1e-5)
    bad = vis.copy()
    bad[0, nt // 2 + 2, nt // 2 + 1] += 5.0
    assert not plan.check_hermitian(torch.from_numpy(bad[None]).cuda(), 1e-5)
    plan.close()


@pytest.mark.parametrize("precision,multires", [(1, True), (0, False)])
def test_merged_plans_equal_one_plan(precision, multires):
    """The exchange step of a channel cube split over ranks, on one GPU: two
    plans accumulate disjoint channel blocks (nu3 split between them), plan A
    imports A's + B's raw collapse sums and sampling (bs_delta_export /
    bs_delta_import, as merge_collapse would after an all-reduce); its folded
    plane and Eq. (dft) equal those of one plan that accumulated every block,
    to FP64 rounding (the atomics add in another order)."""
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    from paper_2506_10526_gb300.sharding import blocks_of
    nt, nc = 40, 12
    edges = synth.edges_log(5, 1.5, 19.0)
    vis = torch.from_numpy(synth.sky_visibilities(nt, nc, seed=93)[None]).cuda()
    flags = np.zeros(nc, np.uint8)
    flags[5] = 1
    jobs = blocks_of(nc, 8, 4)
    plans = [bs.Plan(nt, nc, edges, precision=precision, multires=multires) for _ in range(3)]
    for pl in plans:
        pl.grid_load(vis, chan_flags=flags)
    for k, blk in enumerate(jobs):
        plans[k % 2].mabs(block=blk, accumulate=True)
        plans[2].mabs(block=blk, accumulate=True)
    sa, na = plans[0].delta_export()
    sb, nb_ = plans[1].delta_export()
    assert np.any(na != 0) and np.any(nb_ != 0)
    plans[0].delta_import(sa + sb, na + nb_)
    n2 = 2 * nc - 1
    out = []
    for pl in (plans[0], plans[2]):
        dd = torch.empty((1, pl.ntrip, n2, n2), dtype=torch.float64, device="cuda")
        b3 = torch.empty((1, pl.ntrip, nc, nc), dtype=torch.float64, device="cuda")
        pl.mabs_delta(dd)
        pl.bs3d(b3)
        torch.cuda.synchronize()
        out.append((dd.cpu().numpy(), b3.cpu().numpy(), pl.counts()[1]))
    (d0, b0, c0), (d1, b1, c1) = out
    np.testing.assert_array_equal(c0, c1)
    assert np.array_equal(np.isnan(d0), np.isnan(d1))
    ok = ~np.isnan(d1)
    assert np.abs(d0[ok] - d1[ok]).max() <= 1e-11 * np.abs(d1[ok]).max()
    assert np.abs(b0 - b1).max() <= 1e-5 * max(np.abs(b1).max(), 1e-300)  # FP32 transforms
    # add mode: import B's sums on top of A's own
    plans[1].delta_import(sa, na, add=True)
    dd = torch.empty((1, plans[1].ntrip, n2, n2), dtype=torch.float64, device="cuda")
    plans[1].mabs_delta(dd)
    torch.cuda.synchronize()
    d2 = dd.cpu().numpy()
    assert np.array_equal(np.isnan(d2), np.isnan(d1))
    assert np.abs(d2[ok] - d1[ok]).max() <= 1e-11 * np.abs(d1[ok]).max()
    for pl in plans:
        pl.close()


@pytest.mark.parametrize("nc,block", [(24, None), (48, (0, 4, 0, 4, 0, 4)), (96, (0, 40, 8, 48, 0, 96)),
                                      (12, None), (16, (2, 6, 0, 16, 3, 9)),
                                      (540, (0, 8, 0, 8, 0, 16)), (675, (3, 11, 0, 8, 100, 116)),
                                      (729, (0, 8, 0, 8, 0, 8)), (750, (0, 16, 0, 8, 0, 8))])
def test_delay_transform_against_oracle(nc, block):
    """Eq. (dft) of the library's own folded planes against the oracle's
    transform of the same planes: channel counts with a register FFT (24, 48,
    96, 16; 540, 675, 729, 750 with radix-3 and -5 factors) and one without
    (12), whole-cube and partial channel blocks (rows of the periodic
    placement with nothing sampled), non-unit scale."""
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt, r, rp, dnu = 32, 900.0, 1.2, 0.16
    edges = synth.edges_linear(4, 15)
    vis = synth.sky_visibilities(nt, nc, seed=900 + nc)
    plan = bs.Plan(nt, nc, edges, precision=0, r=r, rprime=rp, dnu_c=dnu)
    plan.grid_load(torch.from_numpy(vis[None]).cuda())
    if block is None:
        plan.mabs(accumulate=True)
    else:
        plan.mabs(block=block, accumulate=True)
    n2 = 2 * nc - 1
    dd = torch.empty((1, plan.ntrip, n2, n2), dtype=torch.float64, device="cuda")
    b3 = torch.empty((1, plan.ntrip, nc, nc), dtype=torch.float64, device="cuda")
    plan.mabs_delta(dd)
    plan.bs3d(b3)
    tri, _ = plan.counts()
    torch.cuda.synchronize()
    want = oracle.delay_dft(dd[0].cpu().numpy(), nc, r, rp, dnu).real
    got = b3[0].cpu().numpy()
    for k in range(plan.ntrip):
        if tri[k] == 0:
            assert np.all(got[k] == 0.0)
            continue
        err = np.abs(got[k] - want[k]).max() / np.abs(want[k]).max()
        assert err < TOL_FP32, (k, err)
    plan.close()
