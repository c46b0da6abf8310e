"""Per-channel sampling N_g(nu) on the GPU against the FP64 oracle: the
sampling differs between channels (flags per baseline), so the denominator
of Eq. (estimator_t) depends on the channel triple.  The library evaluates
the denominators as the I-field triple sums of the occupancy masks, like the
numerators; checked here on the full cube (per-entry ratio), the folded
collapse (the ratio of the summed numerators and denominators, which the
oracle pins to the mean of the estimates for one sampling grid) and
Eq. (dft) of it, for every precision; and end to end from raw baselines with
per-baseline flags through the gridding kernel.  Error measure as elsewhere:
|B_gpu - B_fp64| / B_abs with B_abs the same estimator on |V|."""
import numpy as np
import pytest

import oracle
import synth
from oracle import gridding as gr

pytestmark = pytest.mark.gpu

TOL = {0: 1e-5, 1: 1e-3, 2: 1e-4}


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _occupancy(nc, nt, seed):
    """N_g(nu) in {0, .., 3}, symmetric in U for each channel, varying with nu."""
    r = synth.rng(seed)
    n = r.integers(0, 4, size=(nc, nt, nt)).astype(np.float32)
    n[:, 1:, 1:] = np.maximum(n[:, 1:, 1:], n[:, 1:, 1:][:, ::-1, ::-1])
    return n


def _gpu(vis, edges, ngrid, precision, multires, flags=None, norm_A=1.0):
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    batch, nc, nt, _ = vis.shape
    plan = bs.Plan(nt, nc, edges, precision=precision, multires=multires, batch=batch,
                   chan_sampling=True, norm_A=norm_A)
    plan.grid_load(torch.from_numpy(np.ascontiguousarray(vis.astype(np.complex64))).cuda(),
                   ngrid=torch.from_numpy(ngrid).cuda(), chan_flags=flags)
    full = torch.empty((batch, plan.ntrip, nc, nc, nc), dtype=torch.float64, device="cuda")
    plan.mabs(out_full=full, accumulate=True)
    n2 = 2 * nc - 1
    dd = torch.empty((batch, plan.ntrip, n2, n2), dtype=torch.float64, device="cuda")
    plan.mabs_delta(dd)
    b3 = torch.empty((batch, plan.ntrip, nc, nc), dtype=torch.float64, device="cuda")
    plan.bs3d(b3)
    b3c = torch.empty((batch, plan.n_closable, nc, nc), dtype=torch.float64, device="cuda")
    plan.bs3d_closable(b3c)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in dict(full=full, delta=dd, b3=b3, b3c=b3c).items()}
    out["T"], _ = plan.counts()
    plan.close()
    return out


def _check(out, b, vis, edges, ngrid, flags, precision, label, norm_A=1.0):
    nc = vis.shape[0]  # vis: [nc, nt, nt] of one realisation
    ref = oracle.mabs_full(vis.astype(np.complex128), edges, ngrid=ngrid, chan_flags=flags,
                           norm_A=norm_A)
    rab = oracle.mabs_full(np.abs(vis).astype(np.complex128), edges, ngrid=ngrid,
                           chan_flags=flags, norm_A=norm_A)
    B, babs = ref["B"].real, rab["B"].real
    ok = ~np.isnan(B)
    assert np.array_equal(np.isnan(out["full"][b]), ~ok)
    e_full = np.max(np.abs(out["full"][b][ok] - B[ok]) / babs[ok])
    R = oracle.collapse_fold_ratio(ref["num"], ref["den"], norm_A=norm_A).real
    Rabs = oracle.collapse_fold_ratio(rab["num"], rab["den"], norm_A=norm_A).real
    keep = ref["T"] > 0
    okd = ~np.isnan(R[keep])
    assert np.array_equal(np.isnan(out["delta"][b][keep]), ~okd)
    e_delta = np.max(np.abs(out["delta"][b][keep][okd] - R[keep][okd]) / Rabs[keep][okd])
    b3 = oracle.delay_dft(np.nan_to_num(R), nc).real
    scale = np.abs(oracle.delay_dft(np.nan_to_num(Rabs), nc)).max(axis=(-1, -2), keepdims=True)
    e3 = np.max(np.abs(out["b3"][b][keep] - b3[keep]) / scale[keep])
    np.testing.assert_array_equal(out["b3c"][b], out["b3"][b][np.flatnonzero(out["T"] > 0)])
    # the denominators really differ between channel triples
    den = ref["den"][keep]
    assert np.any(np.nanstd(np.where(den > 0, den, np.nan), axis=(1, 2, 3)) > 0)
    print(f"{label}: full {e_full:.2e}, collapse {e_delta:.2e}, Eq. (dft) {e3:.2e}")
    tol = TOL[precision]
    # a full-cube entry is the ratio of two triple sums, each rounded at the
    # contraction's precision: the numerator's error scales with B_abs, the
    # denominator's (occupancy fields) adds its own, so the entry is held to
    # twice the single-sum tolerance; the collapse and Eq. (dft) to the tolerance
    assert e_full < 2 * tol and e_delta < tol and e3 < tol


@pytest.mark.parametrize("precision,multires", [(0, False), (0, True), (1, True), (2, True)])
def test_per_channel_sampling_against_oracle(precision, multires):
    nt, nc = 32, 6
    edges = synth.edges_log(5, 1.5, 15.0)
    vis = np.stack([synth.sky_visibilities(nt, nc, seed=s) for s in (601, 602)])
    ngrid = _occupancy(nc, nt, 603)
    flags = np.zeros(nc, np.uint8)
    flags[3] = 1
    out = _gpu(vis, edges, ngrid, precision, multires, flags=flags, norm_A=1.7)
    Tgeo = oracle.counts(nt, edges)
    np.testing.assert_array_equal(out["T"], [Tgeo[t] for t in oracle.ring_triples(5)])
    for b in range(2):
        _check(out, b, vis[b], edges, ngrid, flags, precision,
               f"precision {precision} multires {multires} realisation {b}", norm_A=1.7)


def test_gridded_per_baseline_flags_feed_the_estimator():
    """Raw baselines whose flags differ between baselines and channels:
    Eq. (vg) gridding (sums and counts per channel) on the GPU, then a
    per-channel sampling plan, against the oracle estimator on the oracle's
    gridding."""
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt, nc, nbl = 32, 6, 2500
    edges = synth.edges_linear(4, 14)
    r = np.random.default_rng(71)
    uv = r.uniform(-0.5 * nt + 1.0, 0.5 * nt - 1.0, size=(nbl, 2))
    v = (r.normal(size=(nbl, nc)) + 1j * r.normal(size=(nbl, nc))).astype(np.complex64)
    flags = (r.uniform(size=(nbl, nc)) < 0.3).astype(np.uint8)
    plan = bs.Plan(nt, nc, edges)
    vg, ng = plan.grid_visibilities(torch.from_numpy(uv).cuda(), torch.from_numpy(v).cuda(),
                                    torch.from_numpy(flags).cuda(), avg=1, mode=0)
    torch.cuda.synchronize()
    plan.close()
    vg_h, ng_h = vg.cpu().numpy(), ng.cpu().numpy()
    vg_o, ng_o = gr.grid_visibilities(uv, v.astype(np.complex128), flags, nt, avg=1)
    np.testing.assert_array_equal(ng_h, ng_o)
    assert np.any(ng_o[0] != ng_o[1])  # the sampling differs between channels
    out = _gpu(vg_h[None], edges, ng_h, 0, False)
    _check(out, 0, vg_o, edges, ng_o, None, 0, "gridded per-baseline flags")
