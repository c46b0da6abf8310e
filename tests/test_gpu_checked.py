"""The checked build (-DBS_CHECKED, libbs_checked.so): device bounds checks
on the kernels' main global accesses that record a violation and skip the
access instead of faulting.

* the self-test kernel's guarded access: in range nothing is recorded; out of
  range (past the end, negative) the violation is counted with its site,
  index and extent, and the library keeps working;
* tiny grids (8^2, 16^2; plain FP32 and split BF16, one and several image
  sides, register-FFT and Stockham lengths) element by element against the
  FP64 oracle through the checked library, channel-symmetric cubes against
  the ordinary accumulation, then gridding of raw baselines and the
  monopole and multipole binning, with no violation recorded;
* the ordinary library reports that it is not the checked build.
Runs in child processes (BS_LIBRARY selects the library at load time)."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys, numpy as np, torch
    sys.path.insert(0, ROOT)
    import paper_2506_10526_gb300 as bs, synth, oracle
    assert bs.checked_build()
    bs.checked_status(reset=True)
    bs.checked_selftest(16, 3)
    print("INRANGE", bs.checked_status())
    bs.checked_selftest(16, 16)
    print("PAST_END", bs.checked_status())
    bs.checked_selftest(16, -1)
    print("NEGATIVE", bs.checked_status())
    TOL = {0: 1e-5, 1: 1e-3}
    cases = [(8, 4, [1, 2, 3, 4], 0, False), (8, 4, [1, 2, 3, 4], 1, False),
             (16, 6, list(synth.edges_linear(4, 8)), 0, True),
             (16, 16, list(synth.edges_linear(4, 8)), 1, True),
             (16, 12, list(synth.edges_log(3, 1.5, 8.0)), 1, False)]
    worst = 0.0
    for nt, nc, edges, prec, multires in cases:
        vis = synth.sky_visibilities(nt, nc, seed=70 + nt + nc)
        plan = bs.Plan(nt, nc, edges, precision=prec, multires=multires)
        plan.grid_load(torch.from_numpy(vis[None]).cuda())
        full = torch.empty((1, plan.ntrip, nc, nc, nc), dtype=torch.float64, device="cuda")
        plan.mabs(out_full=full, accumulate=True)
        dd = torch.empty((1, plan.ntrip, 2 * nc - 1, 2 * nc - 1), dtype=torch.float64,
                         device="cuda")
        plan.mabs_delta(dd)
        b3 = torch.empty((1, plan.ntrip, nc, nc), dtype=torch.float64, device="cuda")
        plan.bs3d(b3)
        torch.cuda.synchronize()
        ref = oracle.mabs_full(vis.astype(np.complex128), edges)
        babs = oracle.mabs_full(np.abs(vis).astype(np.complex128), edges)["B"].real
        B = ref["B"].real
        ok = ~np.isnan(B)
        got = full[0].cpu().numpy()
        assert np.array_equal(np.isnan(got), ~ok), (nt, nc, "undefined bins differ")
        e_full = np.max(np.abs(got[ok] - B[ok]) / babs[ok]) if ok.any() else 0.0
        bbar, _ = oracle.collapse_fold(B)
        bbar_abs, _ = oracle.collapse_fold(babs)
        keep = ref["T"] > 0
        okd = ~np.isnan(bbar[keep])
        e_d = np.max(np.abs(dd[0].cpu().numpy()[keep][okd] - bbar[keep][okd]) / bbar_abs[keep][okd])
        want3 = oracle.delay_dft(dd[0].cpu().numpy(), nc).real
        g3 = b3[0].cpu().numpy()
        e3 = max(np.abs(g3[k] - want3[k]).max() / np.abs(want3[k]).max() for k in np.flatnonzero(keep))
        print("CASE", nt, nc, prec, multires, e_full, e_d, e3)
        assert e_full < TOL[prec] and e_d < TOL[prec] and e3 < 1e-5, (nt, nc, prec, e_full, e_d, e3)
        plan.close()
    # channel-symmetric cubes (swapped rows, skipped and straddling pair
    # rectangles, the fill-in) against the ordinary accumulation of the same cube
    nt, nc = 16, 40
    edges = list(synth.edges_linear(4, 8))
    vis = torch.from_numpy(synth.sky_visibilities(nt, nc, seed=77)[None]).cuda()
    plan = bs.Plan(nt, nc, edges, precision=1, multires=True)
    for cube in [(0, 40) * 3, (3, 37) * 3]:
        planes = []
        for sym in (True, False):
            plan.grid_load(vis)
            plan.mabs(block=cube, accumulate=True, symmetric=sym)
            dd = torch.empty((1, plan.ntrip, 2 * nc - 1, 2 * nc - 1), dtype=torch.float64,
                             device="cuda")
            plan.mabs_delta(dd)
            planes.append(dd[0].cpu().numpy())
        bound = plan.error_bound()[0][0].cpu().numpy()
        tri, _ = plan.counts()
        assert np.array_equal(np.isnan(planes[0]), np.isnan(planes[1]))
        for k in np.flatnonzero(tri > 0):
            d = np.abs(planes[0][k] - planes[1][k])[~np.isnan(planes[1][k])]
            assert np.all(d <= 2 * bound[k] * (1 + 1e-9)), (cube, k)
        print("SYMMETRIC", cube[:2], "ok")
    plan.close()
    # gridding of raw baselines (the cell checks) and the monopole binning (the
    # bin checks) through the checked library
    from oracle import gridding as gr, monopole as mo
    r = np.random.default_rng(5)
    nt, nc, nbl = 16, 4, 300
    uv = r.uniform(-0.5 * nt - 1.0, 0.5 * nt + 1.0, size=(nbl, 2))
    vis = (r.normal(size=(nbl, nc)) + 1j * r.normal(size=(nbl, nc))).astype(np.complex64)
    plan = bs.Plan(nt, nc, [1.0, 4.0, 8.0])
    vg, ng = plan.grid_visibilities(torch.from_numpy(uv).cuda(), torch.from_numpy(vis).cuda())
    torch.cuda.synchronize()
    vg_o, ng_o = gr.grid_visibilities(uv, vis.astype(np.complex128), None, nt)
    assert np.array_equal(ng.cpu().numpy(), ng_o)
    plan.close()
    nt, nc = 16, 12
    edges = list(synth.edges_linear(4, 8))
    plan = bs.Plan(nt, nc, edges, precision=1)
    plan.grid_load(torch.from_numpy(synth.sky_visibilities(nt, nc, seed=9)[None]).cuda())
    plan.mabs(accumulate=True)
    tri, _ = plan.counts()
    b3 = torch.empty((1, plan.n_closable, nc, nc), dtype=torch.float64, device="cuda")
    plan.bs3d_closable(b3)
    kperp = 2 * np.pi * plan.ring_umean()
    kpar = mo.kpar_axis(nc)
    k1e = np.geomspace(0.5 * kperp.min(), 1.2 * np.sqrt(kperp.max() ** 2 + kpar.max() ** 2), 7)
    _, cnt = plan.bs_monopole(b3, kperp, kpar, k1e, 5, 5)
    _, cntm = plan.bs_multipoles(b3, kperp, kpar, k1e, 5, 5, lmax=2)
    torch.cuda.synchronize()
    assert cnt.sum().item() > 0 and cntm.sum().item() > 0
    plan.close()
    print("AFTER", bs.checked_status())
""").replace("ROOT", repr(ROOT))


def _build_checked():
    sys.path.insert(0, ROOT)
    from paper_2506_10526_gb300 import build
    return build.build(checked=True)


def test_checked_build_records_instead_of_faulting():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _build_checked()
    env = dict(os.environ, BS_LIBRARY="checked")
    r = subprocess.run([sys.executable, "-c", CHILD], capture_output=True, text=True,
                       timeout=900, env=env)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    out = {l.split(" ", 1)[0]: l.split(" ", 1)[1] for l in r.stdout.splitlines() if " " in l}
    print(r.stdout)
    assert "'violations': 0" in out["INRANGE"]
    assert "'violations': 1" in out["PAST_END"] and "'site': 32767" in out["PAST_END"]
    assert "'index': 16" in out["PAST_END"] and "'extent': 16" in out["PAST_END"]
    assert "'violations': 1" in out["NEGATIVE"] and "'index': -1" in out["NEGATIVE"]
    assert "'violations': 0" in out["AFTER"], out["AFTER"]
    assert sum(1 for l in r.stdout.splitlines() if l.startswith("CASE")) == 5


def test_ordinary_build_is_not_checked():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_10526_gb300 as bs
    assert not bs.checked_build()
    with pytest.raises(bs.BsError):
        bs.checked_status()
    with pytest.raises(bs.BsError):
        bs.checked_selftest(16, 3)
