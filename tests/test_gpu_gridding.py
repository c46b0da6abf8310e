"""GPU parity of Eq. (vg) gridding (bs_grid_visibilities) against the oracle
(oracle/gridding.py): counts exact, FP32 atomic sums to rounding, with
random baselines, random flags and 4-channel pre-averaging; and the gridded
mean feeding the estimator end to end against the oracle estimator on the
oracle's own gridding."""
import numpy as np
import pytest

import oracle
import synth
from oracle import gridding as gr

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _baselines(nbl, nin, nt, seed):
    r = np.random.default_rng(seed)
    uv = r.uniform(-0.5 * nt - 1.0, 0.5 * nt + 1.0, size=(nbl, 2))  # some fall outside
    uv[:5] = [[0.5, 0.5], [-0.5, 1.5], [2.5, -3.5], [0.0, 0.0], [-0.5 * nt, 1.0]]
    vis = (r.normal(size=(nbl, nin)) + 1j * r.normal(size=(nbl, nin))).astype(np.complex64)
    return uv, vis


@pytest.mark.parametrize("avg,mode", [(1, 0), (4, 0), (4, 1)])
def test_gridding_matches_oracle(avg, mode):
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt, nc, nbl = 64, 8, 4000
    uv, vis = _baselines(nbl, avg * nc, nt, 17)
    flags = (np.random.default_rng(18).uniform(size=vis.shape) < 0.15).astype(np.uint8)
    plan = bs.Plan(nt, nc, [1.0, 8.0, 16.0])
    vg, ng = plan.grid_visibilities(torch.from_numpy(uv).cuda(), torch.from_numpy(vis).cuda(),
                                    torch.from_numpy(flags).cuda(), avg=avg, mode=mode)
    torch.cuda.synchronize()
    vg_o, ng_o = gr.grid_visibilities(uv, vis.astype(np.complex128), flags, nt, avg=avg)
    got_v, got_n = vg.cpu().numpy(), ng.cpu().numpy()
    absum, _ = gr.grid_visibilities(uv, np.abs(vis).astype(np.complex128), flags, nt, avg=avg)
    if mode == 0:
        np.testing.assert_array_equal(got_n, ng_o)
        assert np.all(np.abs(got_v - vg_o) <= 4e-6 * absum.real + 1e-30)
    else:
        occ = ng_o > 0
        np.testing.assert_array_equal(got_n, occ.astype(np.float32))
        mean = np.where(occ, vg_o / np.maximum(ng_o, 1), 0)
        scale = np.where(occ, absum.real / np.maximum(ng_o, 1), 0)
        assert np.all(np.abs(got_v - mean) <= 4e-6 * scale + 1e-30)
    plan.close()


def test_gridded_mean_feeds_the_estimator():
    """Raw baselines with the coarse-band flag pattern on 32 input channels,
    pre-averaged by 4: gridding (mode 1) + grid_load + the FP32 contraction
    against the oracle estimator on the oracle's gridded mean."""
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt, nc, avg, nbl = 32, 8, 4, 2500
    edges = synth.edges_linear(4, 14)
    uv, vis = _baselines(nbl, avg * nc, nt, 29)
    chan = synth.flag_mask_coarse_band(avg * nc)  # per input channel, every baseline
    flags = np.repeat(chan[None, :], nbl, axis=0).astype(np.uint8)
    plan = bs.Plan(nt, nc, edges)
    vg, occ = plan.grid_visibilities(torch.from_numpy(uv).cuda(), torch.from_numpy(vis).cuda(),
                                     torch.from_numpy(flags).cuda(), avg=avg, mode=1)
    occ0 = occ[0].clone()
    assert torch.equal(occ, occ0.expand_as(occ))  # flags per channel: one occupancy
    plan.grid_load(vg[None], ngrid=occ0)
    full = torch.empty((1, plan.ntrip, nc, nc, nc), dtype=torch.float64, device="cuda")
    plan.mabs(out_full=full, accumulate=False)
    torch.cuda.synchronize()
    vg_o, ng_o = gr.grid_visibilities(uv, vis.astype(np.complex128), flags, nt, avg=avg)
    mean = np.where(ng_o > 0, vg_o / np.maximum(ng_o, 1), 0)
    ngrid = (ng_o[0] > 0).astype(np.float64)
    ref = oracle.mabs_full(mean, edges, ngrid=ngrid)
    babs = oracle.mabs_full(np.abs(mean).astype(np.complex128), edges, ngrid=ngrid)["B"].real
    got = full[0].cpu().numpy()
    ok = ~np.isnan(ref["B"].real)
    assert np.array_equal(np.isnan(got), ~ok)
    e = np.max(np.abs(got[ok] - ref["B"].real[ok]) / babs[ok])
    print(f"gridded estimator: max kappa-normalised error {e:.2e}")
    assert e < 1e-5
    plan.close()
