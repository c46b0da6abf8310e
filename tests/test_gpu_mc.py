"""Batched Monte Carlo (bs_mc_*): two shape groups of uneven sizes, several
runs, per-bin Welford mean and variance of the collapsed plane and the 3D
bispectrum against numpy statistics of the FP64 oracle evaluated on every
realisation; graph replay against eager runs."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

GROUPS = [dict(nt=32, nchan=8, edges=list(synth.edges_linear(4, 16)), batch=3),
          dict(nt=40, nchan=6, edges=list(synth.edges_log(5, 1.5, 19.0)), batch=2, multires=True)]


def _realisation(g, k):
    spec = GROUPS[g]
    return synth.sky_visibilities(spec["nt"], spec["nchan"], 7000 + 100 * g + k)


def _run_ensemble(runs, use_graph, precision=1):
    import torch
    import paper_2506_10526_gb300 as bs
    ens = bs.Ensemble([dict(g, precision=precision) for g in GROUPS])
    bufs = [torch.empty((s["batch"], s["nchan"], s["nt"], s["nt"]), dtype=torch.complex64,
                        device="cuda") for s in GROUPS]
    for g in range(len(GROUPS)):
        ens.set_input(g, bufs[g])
    for r in range(runs):
        for g, spec in enumerate(GROUPS):
            v = np.stack([_realisation(g, r * spec["batch"] + b) for b in range(spec["batch"])])
            bufs[g].copy_(torch.from_numpy(v))
        ens.run(use_graph=use_graph)
    out = [(ens.stats(g, 0), ens.stats(g, 1)) for g in range(len(GROUPS))]
    ens.close()
    return out


@pytest.mark.parametrize("precision", [1, 2])  # split BF16, split FP16
def test_mc_statistics_match_oracle_and_graph_replay(precision):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    runs = 3
    eager = _run_ensemble(runs, use_graph=False, precision=precision)
    graph = _run_ensemble(runs, use_graph=True, precision=precision)
    for g, spec in enumerate(GROUPS):
        n = runs * spec["batch"]
        planes, b3s, abs_planes = [], [], []
        for k in range(n):
            vis = _realisation(g, k).astype(np.complex128)
            res = oracle.mabs_full(vis, spec["edges"])
            bbar, _ = oracle.collapse_fold(res["B"].real)
            planes.append(bbar)
            b3s.append(oracle.delay_dft(bbar, spec["nchan"]).real)
            babs = oracle.mabs_full(np.abs(vis), spec["edges"])["B"].real
            abs_planes.append(oracle.collapse_fold(babs)[0])
        planes, b3s = np.array(planes), np.array(b3s)
        # undefined bins are NaN in every realisation (geometry and sampling alike)
        scale = np.max(np.array(abs_planes), axis=0)
        for which, ref in ((0, planes), (1, b3s)):
            (mean_e, var_e, n_e) = eager[g][which]
            (mean_g, var_g, n_g) = graph[g][which]
            assert n_e == n and n_g == n
            want_m = ref.mean(axis=0)
            want_v = ref.var(axis=0, ddof=1)
            ok = ~np.isnan(want_m)
            assert np.array_equal(np.isnan(mean_e), np.isnan(want_m))
            if which == 0:
                tol = 1e-3 * scale[ok]
            else:
                tol = 1e-3 * np.abs(np.array([oracle.delay_dft(a, spec["nchan"]) for a in abs_planes])).max()
            assert np.all(np.abs(mean_e[ok] - want_m[ok]) <= tol)
            dv = np.abs(var_e[ok] - want_v[ok])
            assert np.all(dv <= 2 * np.sqrt(want_v[ok]) * tol + tol ** 2 + 1e-300)
            # graph replay runs the same launches
            np.testing.assert_allclose(mean_g[ok], mean_e[ok], rtol=1e-9,
                                       atol=1e-12 * np.nanmax(np.abs(mean_e)))


def test_mc_autotuner_cache(tmp_path):
    """The autotuner times its candidates, writes the choice to a JSON cache,
    and a second ensemble of the same shapes reuses the cached choice;
    tuning runs do not count as realisations."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import json
    import paper_2506_10526_gb300 as bs
    cache = tmp_path / "tune.json"
    chosen = []
    for _ in range(2):
        ens = bs.Ensemble(GROUPS)
        bufs = []
        for g, s in enumerate(GROUPS):
            v = np.stack([_realisation(g, b) for b in range(s["batch"])])
            bufs.append(torch.from_numpy(v).cuda())
            ens.set_input(g, bufs[-1])
        chosen.append(ens.autotune(cache))
        mean, var, n = ens.stats(0, 0)
        assert n == 0
        ens.run()
        mean, var, n = ens.stats(0, 0)
        assert n == GROUPS[0]["batch"]
        ens.close()
    assert chosen[0] == chosen[1] and chosen[0] in (1, 2, 4, 8, 16)
    data = json.loads(cache.read_text())
    entry = list(data.values())[0]
    assert len(data) == 1 and entry["tiles_per_sm"] == chosen[0] and entry["order"] in (0, 1)


def _block_collapse(B, blk):
    """Folded mean of the full cube B [ntrip, nc, nc, nc] over the valid channel
    triples of a block (the collapse of Section 3.2 restricted to the block)."""
    ntrip, nc = B.shape[0], B.shape[1]
    n2 = 2 * nc - 1
    s = np.zeros((ntrip, n2, n2))
    c = np.zeros((ntrip, n2, n2))
    for n1 in range(blk[0], blk[1]):
        for n2_ in range(blk[2], blk[3]):
            for n3 in range(blk[4], blk[5]):
                v = B[:, n1, n2_, n3]
                ok = ~np.isnan(v)
                s[ok, n1 - n3 + nc - 1, n2_ - n3 + nc - 1] += v[ok]
                c[ok, n1 - n3 + nc - 1, n2_ - n3 + nc - 1] += 1
    sf, cf = oracle.fold_plane(s), oracle.fold_plane(c)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(cf > 0, sf / np.where(cf > 0, cf, 1), np.nan)


def test_mc_declared_block_subset_and_tile_order():
    """A declared channel block per group (a subset of each realisation's
    tiles): the ensemble mean of the collapsed plane equals the oracle's
    collapse restricted to that block; the autotuner's choice of K extent and
    tile order is reported, and a run with the other tile order gives the
    same statistics."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_10526_gb300 as bs
    blk = (1, 6, 0, 5, 2, 8)
    means = []
    for order in (0, 1):
        ens = bs.Ensemble(GROUPS)
        bufs = []
        for g, spec in enumerate(GROUPS):
            v = np.stack([_realisation(g, b) for b in range(spec["batch"])])
            bufs.append(torch.from_numpy(v).cuda())
            ens.set_input(g, bufs[-1])
        ens.set_block(0, blk)
        if order == 0:
            ens.autotune()
            tps, ordr = ens.tuning()
            assert tps in (1, 2, 4, 8, 16) and ordr in (0, 1)
        ens.run(use_graph=True)
        means.append(ens.stats(0, 0))
        ens.close()
    spec = GROUPS[0]
    planes = []
    for k in range(spec["batch"]):
        res = oracle.mabs_full(_realisation(0, k).astype(np.complex128), spec["edges"])
        planes.append(_block_collapse(res["B"].real, blk))
    want = np.mean(planes, axis=0)
    mean, _, n = means[0]
    assert n == spec["batch"]
    assert np.array_equal(np.isnan(mean), np.isnan(want))
    ok = ~np.isnan(want)
    assert np.abs(mean[ok] - want[ok]).max() <= 1e-3 * np.abs(want[ok]).max()
    np.testing.assert_allclose(means[1][0][ok], mean[ok], rtol=1e-9,
                               atol=1e-12 * np.abs(mean[ok]).max())


def test_mc_checkpoint_and_resume(tmp_path):
    """A run interrupted after three Monte Carlo steps and resumed from its
    checkpoint in a new ensemble (skies drawn on the GPU, the generator's
    realisation counter carried in the checkpoint) ends with the statistics of
    an uninterrupted five-step run."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_10526_gb300 as bs
    groups = [dict(g, precision=1) for g in GROUPS]

    def make():
        ens = bs.Ensemble(groups)
        gens = [bs.SkyGenerator(g["nt"], g["nchan"], max_batch=g["batch"]) for g in groups]
        bufs = [torch.empty((g["batch"], g["nchan"], g["nt"], g["nt"]), dtype=torch.complex64,
                            device="cuda") for g in groups]
        for k, b in enumerate(bufs):
            ens.set_input(k, b)
        return ens, gens, bufs

    def step(ens, gens, bufs, counter):
        for k, g in enumerate(groups):
            gens[k].generate(123, counter * g["batch"], out=bufs[k])
        ens.run(use_graph=True)
        return counter + 1

    ens, gens, bufs = make()
    c = 0
    for _ in range(5):
        c = step(ens, gens, bufs, c)
    want = [(ens.stats(g, 0), ens.stats(g, 1)) for g in range(len(groups))]
    ens.close()
    ens, gens, bufs = make()
    c = 0
    for _ in range(3):
        c = step(ens, gens, bufs, c)
    path = tmp_path / "mc.ckpt"
    ens.checkpoint(path, counter=c)
    ens.close()
    ens, gens2, bufs = make()
    c = ens.restore(path)
    assert c == 3
    for _ in range(2):
        c = step(ens, gens2, bufs, c)
    got = [(ens.stats(g, 0), ens.stats(g, 1)) for g in range(len(groups))]
    ens.close()
    for (w0, w1), (g0, g1) in zip(want, got):
        for (mw, vw, nw), (mg, vg, ng) in ((w0, g0), (w1, g1)):
            assert nw == ng == 5 * (nw // 5)
            ok = ~np.isnan(mw)
            assert np.array_equal(ok, ~np.isnan(mg))
            scale = np.abs(mw[ok]).max()
            assert np.abs(mg[ok] - mw[ok]).max() <= 1e-9 * scale
            okv = ~np.isnan(vw)
            assert np.abs(vg[okv] - vw[okv]).max() <= 1e-8 * np.abs(vw[okv]).max()
    # a checkpoint of other shapes is refused
    other = bs.Ensemble([dict(GROUPS[0], precision=1)])
    with pytest.raises(bs.BsError):
        other.restore(path)
    other.close()


@pytest.mark.parametrize("precision", [1, 2])
def test_mc_channel_symmetric_cubes_match_the_plan(precision):
    """Groups whose channel block is a cube of 64 channels or more contract
    one ordering of a repeated ring's channels and fill in the other: a full
    72-channel cube, a 64-channel sub-cube (bs_mc_set_block) and an ordinary
    24-channel group in one persistent launch.  The ensemble mean of the
    collapsed plane equals the mean of the ordinary plan path on the same
    realisations within the error bound, and so does the graph replay (its
    shared-memory FP32 reductions may add in another order)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2506_10526_gb300 as bs
    edges = list(synth.edges_linear(4, 15))
    specs = [dict(nt=32, nchan=72, edges=edges, batch=2, multires=True),
             dict(nt=32, nchan=80, edges=edges, batch=1, multires=True),
             dict(nt=32, nchan=24, edges=edges, batch=2, multires=True)]
    blocks = [None, (8, 72) * 3, None]
    vis = [np.stack([synth.sky_visibilities(s["nt"], s["nchan"], 8000 + 10 * g + b)
                     for b in range(s["batch"])]) for g, s in enumerate(specs)]
    means = []
    for use_graph in (False, True):
        ens = bs.Ensemble([dict(s, precision=precision) for s in specs])
        bufs = [torch.from_numpy(v).cuda() for v in vis]
        for g in range(len(specs)):
            ens.set_input(g, bufs[g])
            if blocks[g] is not None:
                ens.set_block(g, blocks[g])
        ens.run(use_graph=False)
        if use_graph:
            ens.reset()
            ens.run(use_graph=True)
        means.append([ens.stats(g, 0)[0] for g in range(len(specs))])
        ens.close()
    for g, s in enumerate(specs):
        nc = s["nchan"]
        planes, bounds = [], []
        for b in range(s["batch"]):
            plan = bs.Plan(s["nt"], nc, edges, precision=precision, multires=True)
            plan.grid_load(torch.from_numpy(vis[g][b][None]).cuda())
            plan.mabs(block=blocks[g], accumulate=True)
            dd = torch.empty((1, plan.ntrip, 2 * nc - 1, 2 * nc - 1), dtype=torch.float64,
                             device="cuda")
            plan.mabs_delta(dd)
            bounds.append(plan.error_bound()[0][0].cpu().numpy())
            planes.append(dd[0].cpu().numpy())
            plan.close()
        want = np.mean(planes, axis=0)
        beta = 2 * np.mean(bounds, axis=0) * (1 + 1e-9)
        ok = ~np.isnan(want)
        for got in (means[0][g], means[1][g]):
            assert np.array_equal(np.isnan(got), np.isnan(want)), g
            for k in range(want.shape[0]):
                assert np.all(np.abs(got[k] - want[k])[ok[k]] <= beta[k]), (g, k)
