"""The error bound every estimate carries (bs_mabs_error_bound) against the
actual error of the GPU estimates with respect to the FP64 oracle.

* Coverage: for every ring triple the bound beta must exceed
  |B_gpu - B_fp64| on every entry of the full cube and of the folded,
  collapsed plane (the oracle's own FP64 rounding, ~1e-13 of B_abs, is
  allowed on top).  The ratio error / beta is printed: the bound is
  worst-case, so it sits well above the measured error.
* relerr: the per-bin relative bound equals beta / |B| of the plane it was
  given, in the full and the closable layouts.
* The relative-error rule for well-conditioned bins: with B_abs the
  estimator evaluated by the oracle on |V| and kappa = B_abs / |B|, every bin
  with kappa u <= tol / 10 must have |B_gpu - B_fp64| / |B| <= tol, for the
  unit u of the arithmetic (2^-24 FP32, 2^-17 split BF16, 2^-22 split FP16)
  and the mode's tolerance (1e-5, 1e-3, 1e-4); the kappa distribution is
  printed."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-3, 2: 1e-4}
UNIT = {0: 2.0 ** -24, 1: 2.0 ** -17, 2: 2.0 ** -22}


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _gpu(vis, edges, precision, multires, flags=None, ngrid=None, general=False):
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    if vis.ndim == 3:
        vis = vis[None]
    batch, nc, nt, _ = vis.shape
    plan = bs.Plan(nt, nc, edges, precision=precision, multires=multires, batch=batch,
                   general=general)
    gd = None if ngrid is None else torch.from_numpy(ngrid.astype(np.float32)).cuda()
    plan.grid_load(torch.from_numpy(np.ascontiguousarray(vis.astype(np.complex64))).cuda(),
                   ngrid=gd, chan_flags=flags)
    ct = torch.complex128 if general else torch.float64
    full = torch.empty((batch, plan.ntrip, nc, nc, nc), dtype=ct, device="cuda")
    plan.mabs(out_full=full, accumulate=True)
    n2 = 2 * nc - 1
    dd = torch.empty((batch, plan.ntrip, n2, n2), dtype=ct, device="cuda")
    plan.mabs_delta(dd)
    dc = torch.empty((batch, plan.n_closable, n2, n2), dtype=ct, device="cuda")
    plan.mabs_delta_closable(dc)
    bound, rel = plan.error_bound(dd)
    bound2, relc = plan.error_bound(dc, closable=True)
    torch.cuda.synchronize()
    tri, _ = plan.counts()
    out = {k: v.cpu().numpy() for k, v in
           dict(full=full, delta=dd, closable=dc, bound=bound, rel=rel, bound2=bound2,
                relc=relc).items()}
    out["T"] = tri
    plan.close()
    return out


def _check(out, b, ref, babs, precision, label):
    B = ref["B"].real
    T = ref["T"]
    beta = out["bound"][b]
    np.testing.assert_array_equal(np.isnan(beta), T == 0)
    np.testing.assert_array_equal(out["bound2"][b], beta)
    ok = ~np.isnan(B)
    err = np.abs(out["full"][b] - B)
    slack = 1e-13 * babs
    cover = err[ok] <= (np.broadcast_to(beta[:, None, None, None], B.shape)[ok] + slack[ok])
    ratio = err[ok] / np.broadcast_to(beta[:, None, None, None], B.shape)[ok]
    assert cover.all(), (label, ratio.max())
    # folded, collapsed plane
    bbar, _ = oracle.collapse_fold(B)
    bbar_abs, _ = oracle.collapse_fold(babs)
    okd = ~np.isnan(bbar)
    errd = np.abs(out["delta"][b] - bbar)
    betad = np.broadcast_to(beta[:, None, None], bbar.shape)
    assert np.all(errd[okd] <= betad[okd] + 1e-13 * bbar_abs[okd]), label
    # relerr = beta / |B| on the plane it was given, in both layouts
    with np.errstate(divide="ignore", invalid="ignore"):
        want_rel = betad / np.abs(out["delta"][b])
    np.testing.assert_allclose(out["rel"][b][okd], want_rel[okd], rtol=1e-15)
    assert np.all(np.isnan(out["rel"][b][~okd]))
    clos = np.flatnonzero(T > 0)
    np.testing.assert_array_equal(out["relc"][b], out["rel"][b][clos])
    # well-conditioned bins: relative error within the tolerance
    with np.errstate(divide="ignore", invalid="ignore"):
        kappa = babs[ok] / np.abs(B[ok])
        erel = err[ok] / np.abs(B[ok])
    tol, u = TOL[precision], UNIT[precision]
    good = kappa * u <= tol / 10
    q = np.percentile(kappa[np.isfinite(kappa)], [50, 90, 99])
    print(f"{label}: error/bound max {ratio.max():.2e} median {np.median(ratio):.2e}; kappa "
          f"p50 {q[0]:.3g} p90 {q[1]:.3g} p99 {q[2]:.3g}; {good.sum()} of {good.size} bins "
          f"well-conditioned, max e_rel there {erel[good].max() if good.any() else 0:.2e}")
    assert good.sum() > 0
    assert np.all(erel[good] <= tol), (label, erel[good].max())
    assert np.all(err[ok] / babs[ok] <= tol)


@pytest.mark.parametrize("precision,multires", [(0, False), (0, True), (1, True), (1, False), (2, True)])
@pytest.mark.parametrize("flagged", [False, True])
def test_bound_covers_the_error_tiny_config(precision, multires, flagged):
    """64^2 grid, 16 channels, 8 linear rings (with and without the
    coarse-band flags): every entry of the full cube and the folded plane."""
    nt, nc = 64, 16
    edges = synth.edges_linear(8, 32)
    vis = synth.sky_visibilities(nt, nc, seed=1001)
    flags = synth.flag_mask_coarse_band(nc) if flagged else None
    out = _gpu(vis, edges, precision, multires, flags=flags)
    ref = oracle.mabs_full(vis.astype(np.complex128), edges, chan_flags=flags)
    babs = oracle.mabs_full(np.abs(vis).astype(np.complex128), edges, chan_flags=flags)["B"].real
    np.testing.assert_array_equal(out["T"], ref["T"])
    _check(out, 0, ref, babs, precision, f"p{precision} mr{int(multires)} fl{int(flagged)}")


@pytest.mark.parametrize("precision,multires", [(0, False), (1, True), (2, True)])
def test_bound_covers_the_error_ragged_occupancy_batch(precision, multires):
    """40^2 grid, 11 channels, log rings, N_g in {0, 1, 2, 3}, one flagged
    channel, two realisations of different amplitude."""
    nt, nc = 40, 11
    edges = synth.edges_log(5, 1.5, 19.0)
    v = np.stack([synth.sky_visibilities(nt, nc, seed=s) for s in (42, 44)])
    v[1] *= 50.0
    r = synth.rng(43)
    ngrid = r.integers(0, 4, size=(nt, nt)).astype(np.float32)
    ngrid[1:, 1:] = np.maximum(ngrid[1:, 1:], ngrid[1:, 1:][::-1, ::-1])
    flags = np.zeros(nc, np.uint8)
    flags[4] = 1
    out = _gpu(v, edges, precision, multires, flags=flags, ngrid=ngrid)
    for b in range(2):
        ref = oracle.mabs_full(v[b].astype(np.complex128), edges, chan_flags=flags, ngrid=ngrid)
        babs = oracle.mabs_full(np.abs(v[b]).astype(np.complex128), edges, chan_flags=flags,
                                ngrid=ngrid)["B"].real
        _check(out, b, ref, babs, precision, f"ragged p{precision} realisation {b}")


@pytest.mark.parametrize("precision,multires", [(0, False), (0, True), (1, True), (2, True)])
def test_bound_covers_the_error_general_input(precision, multires):
    """General (non-Hermitian) input: visibilities with no symmetry on an
    asymmetric sampling grid, one flagged channel, two realisations of
    different amplitude.  The estimates are complex, combined from four real
    evaluations; the bound on the modulus of the complex error must cover
    every entry of the full cube and of the folded plane, and relerr is the
    bound over |B| in both layouts."""
    nt, nc = 32, 6
    edges = synth.edges_log(5, 1.5, 15.0)
    r = synth.rng(601)
    v = r.standard_normal((2, nc, nt, nt)) + 1j * r.standard_normal((2, nc, nt, nt))
    v[1] *= 30.0
    v = v.astype(np.complex64)
    ngrid = r.integers(0, 4, size=(nt, nt)).astype(np.float32)  # no symmetry
    flags = np.zeros(nc, np.uint8)
    flags[2] = 1
    out = _gpu(v, edges, precision, multires, flags=flags, ngrid=ngrid, general=True)
    for b in range(2):
        ref = oracle.mabs_full(v[b].astype(np.complex128), edges, ngrid=ngrid, chan_flags=flags)
        babs = oracle.mabs_full(np.abs(v[b]).astype(np.complex128), edges, ngrid=ngrid,
                                chan_flags=flags)["B"].real
        B = ref["B"]
        assert np.nanmax(np.abs(B.imag)) > 0.1 * np.nanmax(np.abs(B.real))  # really complex
        beta = out["bound"][b]
        np.testing.assert_array_equal(np.isnan(beta), ref["T"] == 0)
        np.testing.assert_array_equal(out["bound2"][b], beta)
        ok = ~np.isnan(B)
        err = np.abs(out["full"][b] - B)
        bb = np.broadcast_to(beta[:, None, None, None], B.shape)
        ratio = err[ok] / bb[ok]
        assert np.all(err[ok] <= bb[ok] + 1e-13 * babs[ok]), ratio.max()
        bbar, _ = oracle.collapse_fold(B)
        bbar_abs, _ = oracle.collapse_fold(babs)
        okd = ~np.isnan(bbar)
        errd = np.abs(out["delta"][b] - bbar)
        betad = np.broadcast_to(beta[:, None, None], bbar.shape)
        assert np.all(errd[okd] <= betad[okd] + 1e-13 * bbar_abs[okd])
        with np.errstate(divide="ignore", invalid="ignore"):
            want_rel = betad / np.abs(out["delta"][b])
        np.testing.assert_allclose(out["rel"][b][okd], want_rel[okd], rtol=1e-15)
        assert np.all(np.isnan(out["rel"][b][~okd]))
        clos = np.flatnonzero(ref["T"] > 0)
        np.testing.assert_array_equal(out["relc"][b], out["rel"][b][clos])
        print(f"general p{precision} mr{int(multires)} realisation {b}: error/bound max "
              f"{ratio.max():.2e} median {np.median(ratio):.2e}")


@pytest.mark.parametrize("precision,multires", [(0, False), (0, True), (1, True), (2, True)])
def test_bound_covers_the_error_per_channel_sampling(precision, multires):
    """Per-channel sampling N_g(nu): denominators that depend on the channel
    triple and the ratio-of-sums collapse, two realisations of different
    amplitude, a flagged channel, A != 1.  The per-bin bound of the folded
    plane covers the oracle error on every bin, in the full and the closable
    layout; the ring-triple bound is the largest bin bound; without a plane
    the call is refused."""
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt, nc, A = 32, 6, 1.7
    edges = synth.edges_log(5, 1.5, 15.0)
    vis = np.stack([synth.sky_visibilities(nt, nc, seed=s) for s in (611, 612)])
    vis[1] *= 40.0
    g = synth.rng(613)
    ngrid = g.integers(0, 4, size=(nc, nt, nt)).astype(np.float32)
    ngrid[:, 1:, 1:] = np.maximum(ngrid[:, 1:, 1:], ngrid[:, 1:, 1:][:, ::-1, ::-1])
    flags = np.zeros(nc, np.uint8)
    flags[3] = 1
    plan = bs.Plan(nt, nc, edges, precision=precision, multires=multires, batch=2,
                   chan_sampling=True, norm_A=A)
    plan.grid_load(torch.from_numpy(vis.astype(np.complex64)).cuda(),
                   ngrid=torch.from_numpy(ngrid).cuda(), chan_flags=flags)
    plan.mabs(accumulate=True)
    n2 = 2 * nc - 1
    dd = torch.empty((2, plan.ntrip, n2, n2), dtype=torch.float64, device="cuda")
    plan.mabs_delta(dd)
    dc = torch.empty((2, plan.n_closable, n2, n2), dtype=torch.float64, device="cuda")
    plan.mabs_delta_closable(dc)
    bound, rel = plan.error_bound(dd)
    bound2, relc = plan.error_bound(dc, closable=True)
    with pytest.raises(bs.BsError):
        plan.error_bound()  # the bound is per bin: the plane is required
    torch.cuda.synchronize()
    tri, _ = plan.counts()
    d, bnd, r, bnd2, rc = (x.cpu().numpy() for x in (dd, bound, rel, bound2, relc))
    plan.close()
    clos = np.flatnonzero(tri > 0)
    for b in range(2):
        ref = oracle.mabs_full(vis[b].astype(np.complex128), edges, ngrid=ngrid, chan_flags=flags,
                               norm_A=A)
        rab = oracle.mabs_full(np.abs(vis[b]).astype(np.complex128), edges, ngrid=ngrid,
                               chan_flags=flags, norm_A=A)
        R = oracle.collapse_fold_ratio(ref["num"], ref["den"], norm_A=A).real
        Rabs = oracle.collapse_fold_ratio(rab["num"], rab["den"], norm_A=A).real
        ok = ~np.isnan(R)
        assert np.array_equal(np.isnan(d[b]), ~ok)
        np.testing.assert_array_equal(np.isnan(r[b]), ~ok)
        np.testing.assert_array_equal(np.isnan(bnd[b]), tri == 0)
        err = np.abs(d[b] - R)
        ebin = r[b] * np.abs(d[b])  # the absolute bound of each bin
        ratio = err[ok] / ebin[ok]
        assert np.all(err[ok] <= ebin[ok] + 1e-13 * Rabs[ok]), ratio.max()
        want = np.array([np.max(ebin[t][ok[t]]) if ok[t].any() else 0.0 for t in clos])
        np.testing.assert_allclose(bnd[b][clos], want, rtol=1e-12)
        np.testing.assert_array_equal(rc[b], r[b][clos])
        np.testing.assert_array_equal(bnd2[b], bnd[b])
        print(f"per-channel p{precision} mr{int(multires)} realisation {b}: error/bound max "
              f"{ratio.max():.2e} median {np.median(ratio):.2e}; infinite bins "
              f"{int(np.isinf(ebin[ok]).sum())} of {int(ok.sum())}")
