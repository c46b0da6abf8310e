"""Error-bar surrogate (bs_mlp_*) on the GPU.

* forward and gradient of the network against the FP64 reference
  (oracle/mlp.py) evaluated with the same BF16-rounded weights;
* the 45 bin features against a numpy restatement of their definition;
* the tensor-core kernels against the FP32 SIMT checker;
* accuracy: trained on Monte Carlo variances from 4096 realisations of the
  batched path (skies drawn by the GPU generator, tensor-core training) on
  training flag masks -- a coarse-band family
  (edge widths 0-3, centre on/off) plus random masks -- the predicted sigma
  of every 3D-bispectrum bin on held-out family masks is within 10% (median)
  of a 1024-realisation Monte Carlo, and beats what a 16-realisation Monte
  Carlo gives on those masks."""
import itertools

import numpy as np
import pytest

import oracle
import synth
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

NT, NC = 64, 16
EDGES = list(synth.edges_linear(8, 32))


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("kernels,d", [("tensor", None), ("simt", None), ("tensor", 20),
                                       ("tensor", 64)])
def test_forward_and_gradient_match_fp64_reference(kernels, d):
    """Both kernel sets (BF16 tensor cores with hi / lo activations, FP32 SIMT),
    several input widths (the tensor-core input padding), ragged row counts."""
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    d, w, n = d or bs.MLP_FEATURES, 128, 3000
    r = np.random.default_rng(11)
    x = r.standard_normal((n, d)).astype(np.float32) * 2 + 0.5
    t = (np.sin(x[:, 0]) + 0.3 * x[:, 1] * x[:, 2]).astype(np.float32)
    net = bs.Surrogate(d, w, seed=5)
    net.set_kernels(kernels)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    net.fit_norm(xd, td)
    net.train(xd, td, steps=50, batch=512, lr=1e-3)  # move away from the initial point
    p = net.params().astype(np.float64)
    nw = net.n_weights
    norm = (p[nw:nw + d], p[nw + d:nw + 2 * d], p[nw + 2 * d], p[nw + 2 * d + 1])
    assert np.allclose(norm[0], x.mean(0), rtol=1e-4, atol=1e-4)
    y = net.forward(xd).cpu().numpy()
    y_ref, _ = omlp.forward(p[:nw], x.astype(np.float64), d, w, norm, bf16=True)
    np.testing.assert_allclose(y, y_ref, rtol=1e-4, atol=1e-4 * np.abs(y_ref).max())
    loss, g = net.grad(xd, td)
    loss_ref, g_ref = omlp.loss_and_grad(p[:nw], x.astype(np.float64), t.astype(np.float64), d, w,
                                         norm, bf16=True)
    assert loss == pytest.approx(loss_ref, rel=1e-4)
    np.testing.assert_allclose(g, g_ref, rtol=0, atol=2e-4 * np.abs(g_ref).max())
    net.close()


def test_tensor_and_simt_kernels_agree():
    """The tensor-core forward and gradient against the FP32 SIMT checker on
    the same network: forward to 2e-5 of the output scale, gradients to 2e-4
    of the largest component; training steps with each stay close."""
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    d, n = bs.MLP_FEATURES, 5003
    r = np.random.default_rng(21)
    x = torch.from_numpy(r.standard_normal((n, d)).astype(np.float32)).cuda()
    t = torch.from_numpy(r.standard_normal(n).astype(np.float32)).cuda()
    a, b = bs.Surrogate(d, 128, seed=9), bs.Surrogate(d, 128, seed=9)
    a.set_kernels("tensor")
    b.set_kernels("simt")
    for net in (a, b):
        net.fit_norm(x, t)
    ya, yb = a.forward(x).cpu().numpy(), b.forward(x).cpu().numpy()
    np.testing.assert_allclose(ya, yb, rtol=0, atol=2e-5 * np.abs(yb).max())
    (la, ga), (lb, gb) = a.grad(x, t), b.grad(x, t)
    assert la == pytest.approx(lb, rel=1e-5)
    np.testing.assert_allclose(ga, gb, rtol=0, atol=2e-4 * np.abs(gb).max())
    la = a.train(x, t, steps=20, batch=1024, lr=1e-3)
    lb = b.train(x, t, steps=20, batch=1024, lr=1e-3)
    assert la == pytest.approx(lb, rel=1e-2)
    pa, pb = a.params(), b.params()
    assert np.abs(pa - pb).max() < 1e-3 * np.abs(pb).max()
    with pytest.raises(bs.BsError):
        bs.Surrogate(d, 64, seed=1).set_kernels("tensor")
    a.close()
    b.close()


def _sampling_features(flags):
    """log sum 1/N, sampled fraction, log mean N over the Eq. (dft) square
    (-NC/2 <= d < NC/2) of the folded sampling N of valid channel triples."""
    nn = oracle.fold_plane(oracle.n_nu(1 - flags)).astype(float)
    h = NC // 2
    sq = nn[NC - 1 - h:2 * NC - 1 - h, NC - 1 - h:2 * NC - 1 - h]
    s = sq[sq > 0]
    if s.size == 0:
        return [0.0, 0.0, 0.0]
    return [np.log((1.0 / s).sum()), s.size / sq.size, np.log(s.mean())]


def _features_reference(flags):
    lab = oracle.ring_labels(NT, EDGES)
    u = np.arange(NT) - NT // 2
    uu, vv = np.meshgrid(u, u, indexing="xy")
    umean = np.array([np.hypot(uu, vv)[lab == m].mean() for m in range(len(EDGES) - 1)])
    T = oracle.counts(NT, EDGES)
    trips = oracle.ring_triples(len(EDGES) - 1)
    kp = 2 * np.pi * umean
    h = NC // 2
    rows = []
    frac = flags.mean()
    pos = [flags[np.arange(NC) % 32 == q].mean() if np.any(np.arange(NC) % 32 == q) else 0.0
           for q in range(32)]
    samp = _sampling_features(flags)
    for (i, j, l) in trips:
        for ia in range(NC):
            for ib in range(NC):
                if T[i, j, l] == 0:
                    rows.append([np.nan] * 45)
                    continue
                ka, kb = 2 * np.pi * (ia - h) / NC, 2 * np.pi * (ib - h) / NC
                k = sorted([np.hypot(kp[i], ka), np.hypot(kp[j], kb), np.hypot(kp[l], ka + kb)],
                           reverse=True)
                rows.append([np.log(k[0]), k[1] / k[0], (k[0]**2 + k[1]**2 - k[2]**2) / (2 * k[0] * k[1]),
                             frac, np.log(T[i, j, l]), abs(ka), abs(kb), np.log(kp[i]), np.log(kp[j]),
                             np.log(kp[l])] + pos + samp)
    return np.array(rows)


def test_features_match_definition():
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    flags = np.zeros(NC, np.uint8)
    flags[[0, 1, 8, 15]] = 1
    plan = bs.Plan(NT, NC, EDGES)
    got = plan.mlp_features(flags).cpu().numpy()
    plan.close()
    want = _features_reference(flags)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    np.testing.assert_allclose(got[ok], want[ok], rtol=2e-6, atol=2e-6)


def _masks():
    out = []
    for wl, wh, cen in itertools.product(range(4), range(4), (0, 1)):
        f = np.zeros(NC, np.uint8)
        f[:wl] = 1
        if wh:
            f[NC - wh:] = 1
        if cen:
            f[NC // 2] = 1
        out.append(f)
    return np.array(out)


def _mc_variance(masks, nreal, seed0, batch=64):
    """Per-bin variance of the 3D bispectrum for each mask, from the batched
    Monte Carlo path (all masks share the same sky realisations)."""
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    b = min(batch, nreal)
    ens = bs.Ensemble([dict(nt=NT, nchan=NC, edges=EDGES, batch=b) for _ in masks])
    gen = bs.SkyGenerator(NT, NC, max_batch=b)
    buf = torch.empty((b, NC, NT, NT), dtype=torch.complex64, device="cuda")
    for g, m in enumerate(masks):
        ens.set_input(g, buf)
        ens.set_flags(g, m)
    for r in range(nreal // b):
        gen.generate(seed0, r * b, out=buf)
        ens.run(use_graph=True)
    out = np.array([ens.stats(g, 1)[1].reshape(-1) for g in range(len(masks))])
    gen.close()
    ens.close()
    return out


def _random_masks(n, seed):
    """Random coarse-band-like masks: each channel flagged with a per-mask
    probability drawn from [0, 0.25)."""
    r = np.random.default_rng(seed)
    return np.array([(r.random(NC) < r.uniform(0.0, 0.25)).astype(np.uint8) for _ in range(n)])


def test_surrogate_error_bars_on_held_out_masks():
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    masks = _masks()
    perm = np.random.default_rng(5).permutation(len(masks))
    held, train = masks[perm[:4]], np.concatenate([masks[perm[4:28]], _random_masks(40, 77)])
    var_tr = _mc_variance(train, 4096, 100000)  # training targets from 4096 realisations
    var_ho = _mc_variance(held, 1024, 900000)
    var_16 = _mc_variance(held, 16, 500000, batch=16)
    plan = bs.Plan(NT, NC, EDGES)
    feats = [plan.mlp_features(m) for m in list(train) + list(held)]
    X, Y = [], []
    for f, v in zip(feats[:len(train)], var_tr):
        ok = torch.isfinite(f[:, 0]).cpu().numpy() & np.isfinite(v) & (v > 0)
        X.append(f[torch.from_numpy(ok).cuda()])
        Y.append(torch.from_numpy(np.log(v[ok]).astype(np.float32)).cuda())
    X, Y = torch.cat(X).contiguous(), torch.cat(Y).contiguous()
    net = bs.Surrogate(bs.MLP_FEATURES, 128, seed=3)
    net.fit_norm(X, Y)
    net.train(X, Y, steps=12000, batch=8192, lr=2e-3)
    net.train(X, Y, steps=4000, batch=8192, lr=4e-4)
    err_net, err_16 = [], []
    for f, v, v16 in zip(feats[len(train):], var_ho, var_16):
        ok = torch.isfinite(f[:, 0]).cpu().numpy() & np.isfinite(v) & (v > 0) & np.isfinite(v16)
        pred = net.forward(f[torch.from_numpy(ok).cuda()].contiguous()).cpu().numpy()
        sig_mc = np.sqrt(v[ok])
        err_net.append(np.median(np.abs(np.exp(0.5 * pred) / sig_mc - 1)))
        err_16.append(np.median(np.abs(np.sqrt(v16[ok]) / sig_mc - 1)))
    print("held-out median |sigma_pred/sigma_MC1024 - 1|:", np.round(err_net, 3),
          " 16-realisation MC:", np.round(err_16, 3))
    net.close()
    plan.close()
    assert max(err_net) <= 0.10
    assert np.mean(err_net) < np.mean(err_16)
