"""GPU parity of the binned 3D-bispectrum monopole (bs_bs_monopole) against
the oracle (oracle/monopole.py), which decides bins in FP64 from Eq. (shape).
The kernel decides them in FP32 on squared lengths, so a sample may land in
another bin only when its FP64 k1 lies within a relative REL_K of a k1 edge
or its mu or t within REL_S of a shape edge: the GPU counts must lie between the
samples that are sure of a bin and those that can reach it, and the sums
must match the sure samples' sums up to the ambiguous samples' |values|.
Run on the GPU's own 3D bispectrum and on the binned Eq. (bsana) model; the
ring centres the plan reports against the oracle's; the full MWA-like
geometry."""
import numpy as np
import pytest

import oracle
import synth
from oracle import monopole as mo

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


# the kernel's FP32 rounding bounds, with a factor 2 to spare: k1 (relative)
# 9 u, t 17 u and mu 68 u (u = 2^-24)
REL_K, REL_S = 2e-6, 1e-5


def _planes_trips(tri, nb):
    trips = oracle.ring_triples(nb)
    return [trips[t] for t in np.flatnonzero(tri > 0)]


def _check_interval(c, s, iv, c_fp64, tol, max_amb=0.1):
    """GPU counts c and sums s against the oracle's interval iv; c_fp64 the
    oracle's own counts (reported); tol the rounding allowance of the sums."""
    assert np.all(iv["c_lo"] <= c) and np.all(c <= iv["c_hi"]), "counts outside the interval"
    assert np.all(np.abs(s - iv["s_sure"]) <= iv["s_amb"] + tol), np.abs(s - iv["s_sure"]).max()
    moved = int(np.abs(c - c_fp64).sum())
    print(f"samples {iv['n']}, near an edge {iv['n_amb']}; "
          f"|GPU - FP64| summed over bins {moved}")
    assert iv["n_amb"] < max_amb * iv["n"]


@pytest.mark.parametrize("precision,multires", [(1, True), (0, False)])
def test_monopole_on_estimated_bispectrum(precision, multires):
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt, nc, r, rp, dnu = 64, 24, 900.0, 1.2, 0.16
    edges = synth.edges_log(8, 1.5, 31.0)
    v = np.stack([synth.sky_visibilities(nt, nc, seed=s) for s in (71, 72)])
    plan = bs.Plan(nt, nc, edges, precision=precision, batch=2, r=r, rprime=rp, dnu_c=dnu,
                   multires=multires)
    plan.grid_load(torch.from_numpy(v).cuda())
    plan.mabs(accumulate=True)
    tri, _ = plan.counts()
    ncl = plan.n_closable
    b3 = torch.empty((2, ncl, nc, nc), dtype=torch.float64, device="cuda")
    plan.bs3d_closable(b3)
    umean = plan.ring_umean()
    np.testing.assert_allclose(umean, mo.ring_mean_u(nt, edges), rtol=1e-14)
    kperp = 2 * np.pi * umean / r
    kpar = mo.kpar_axis(nc, rp, dnu)
    k1e = np.geomspace(0.5 * kperp.min(), 1.2 * np.sqrt(kperp.max() ** 2 + kpar.max() ** 2), 13)
    sums, cnt = plan.bs_monopole(b3, kperp, kpar, k1e, 5, 5)
    torch.cuda.synchronize()
    b3h = b3.cpu().numpy()
    trips = _planes_trips(tri, len(edges) - 1)
    _, c_o = mo.bs_monopole(b3h, trips, kperp, kpar, k1e, 5, 5)
    iv = mo.monopole_interval(b3h, trips, kperp, kpar, k1e, 5, 5, REL_K, REL_S)
    c = cnt.cpu().numpy()
    assert c.sum() > 0.5 * ncl * nc * nc  # most samples fall inside the bins
    s = sums.cpu().numpy()
    _check_interval(c, s, iv, c_o, 1e-12 * np.abs(b3h).max() * np.maximum(iv["c_hi"], 1))
    plan.close()


def test_monopole_of_the_analytic_model():
    """NULL values: Eq. (bsana) with P = A k^-2 binned at the same modes."""
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt, nc, r, rp, dnu = 48, 16, 500.0, 0.9, 0.2
    edges = synth.edges_log(6, 1.5, 23.0)
    plan = bs.Plan(nt, nc, edges, precision=1, multires=True, r=r, rprime=rp, dnu_c=dnu)
    plan.grid_load(torch.zeros((1, nc, nt, nt), dtype=torch.complex64, device="cuda"))
    tri, _ = plan.counts()
    kperp = 2 * np.pi * plan.ring_umean() / r
    kpar = mo.kpar_axis(nc, rp, dnu)
    k1e = np.geomspace(0.01, 4.0, 13)
    model = (0.8, 3.0, -2.0)
    sums, cnt = plan.bs_monopole(None, kperp, kpar, k1e, 5, 5, model=model)
    torch.cuda.synchronize()
    trips = _planes_trips(tri, len(edges) - 1)
    s_o, c_o = mo.bs_monopole(None, trips, kperp, kpar, k1e, 5, 5, model=model)
    iv = mo.monopole_interval(None, trips, kperp, kpar, k1e, 5, 5, REL_K, REL_S, model=model)
    s = sums.cpu().numpy()
    _check_interval(cnt.cpu().numpy(), s, iv, c_o, 1e-11 * np.abs(s_o))
    plan.close()


def test_monopole_geometry_full_mwa_size():
    """The 256^2 x 768-channel MWA-like geometry (684 closable ring triples x
    768^2 delay pairs, 4.0e8 samples): bin counts and the binned model
    within the oracle's interval."""
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt, nc = 256, 768
    edges = synth.edges_log(20, 4.41, 128.0)
    r, rp, dnu = 8900.0, 17.0, 0.04
    plan = bs.Plan(nt, nc, edges, precision=1, multires=True, r=r, rprime=rp, dnu_c=dnu)
    plan.grid_load(torch.zeros((1, nc, nt, nt), dtype=torch.complex64, device="cuda"))
    tri, _ = plan.counts()
    kperp = 2 * np.pi * plan.ring_umean() / r
    kpar = mo.kpar_axis(nc, rp, dnu)
    k1e = np.geomspace(2e-3, 10.0, 13)
    model = (1.0, 1.0, -2.0)
    sums, cnt = plan.bs_monopole(None, kperp, kpar, k1e, 5, 5, model=model)
    torch.cuda.synchronize()
    trips = _planes_trips(tri, len(edges) - 1)
    assert len(trips) == 684
    s_o, c_o = mo.bs_monopole_pool(trips, kperp, kpar, k1e, 5, 5, model)
    iv = mo.monopole_interval_pool(trips, kperp, kpar, k1e, 5, 5, model, REL_K, REL_S)
    c = cnt.cpu().numpy()
    print(f"samples binned: {c.sum()} of {len(trips) * nc * nc}; occupied bins {(c > 0).sum()}")
    assert c.sum() > 0.5 * len(trips) * nc * nc
    s = sums.cpu().numpy()
    _check_interval(c, s, iv, c_o, 1e-10 * np.abs(s_o), max_amb=1e-2)
    plan.close()


def test_cylindrical_binning_matches_oracle():
    """(k_par1, k_par2) binning (Section 5, 20 x 20 like Fig. cylbs) of the
    GPU's closable 3D bispectrum, two realisations: counts exact, sums to
    rounding; edges that leave delay indices outside on both ends."""
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt, nc, rp, dnu = 48, 40, 1.1, 0.16
    edges = synth.edges_log(6, 1.5, 23.0)
    v = np.stack([synth.sky_visibilities(nt, nc, seed=s) for s in (81, 82)])
    plan = bs.Plan(nt, nc, edges, precision=1, batch=2, rprime=rp, dnu_c=dnu, multires=True)
    plan.grid_load(torch.from_numpy(v).cuda())
    plan.mabs(accumulate=True)
    b3 = torch.empty((2, plan.n_closable, nc, nc), dtype=torch.float64, device="cuda")
    plan.bs3d_closable(b3)
    kpar = mo.kpar_axis(nc, rp, dnu)
    ke = np.linspace(-0.8 * kpar.max(), 0.8 * kpar.max(), 21)
    sums, cnt = plan.bs_cylindrical(b3, kpar, ke)
    torch.cuda.synchronize()
    b3h = b3.cpu().numpy()
    s_o, c_o = mo.bs_cylindrical(b3h, kpar, ke)
    np.testing.assert_array_equal(cnt.cpu().numpy(), c_o)
    scale = np.abs(b3h).max() * np.maximum(c_o, 1)
    assert np.all(np.abs(sums.cpu().numpy() - s_o) <= 1e-12 * scale)
    plan.close()


def test_monopole_more_realisations_than_one_launch_holds():
    """Ten realisations: the host splits them into launches of at most eight
    (counts taken by the first); every realisation's sums against the oracle."""
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt, nc, batch = 24, 8, 10
    edges = synth.edges_linear(4, 11)
    v = np.stack([synth.sky_visibilities(nt, nc, seed=300 + k) for k in range(batch)])
    plan = bs.Plan(nt, nc, edges, precision=1, batch=batch)
    plan.grid_load(torch.from_numpy(v).cuda())
    plan.mabs(accumulate=True)
    tri, _ = plan.counts()
    b3 = torch.empty((batch, plan.n_closable, nc, nc), dtype=torch.float64, device="cuda")
    plan.bs3d_closable(b3)
    kperp = 2 * np.pi * plan.ring_umean()
    kpar = mo.kpar_axis(nc)
    k1e = np.geomspace(0.5 * kperp.min(), 2 * np.sqrt(kperp.max() ** 2 + 4 * kpar.max() ** 2), 7)
    sums, cnt = plan.bs_monopole(b3, kperp, kpar, k1e, 5, 5)
    torch.cuda.synchronize()
    b3h = b3.cpu().numpy()
    trips = _planes_trips(tri, len(edges) - 1)
    _, c_o = mo.bs_monopole(b3h, trips, kperp, kpar, k1e, 5, 5)
    iv = mo.monopole_interval(b3h, trips, kperp, kpar, k1e, 5, 5, REL_K, REL_S)
    _check_interval(cnt.cpu().numpy(), sums.cpu().numpy(), iv, c_o,
                    1e-12 * np.abs(b3h).max() * np.maximum(iv["c_hi"], 1))
    plan.close()


@pytest.mark.parametrize("nc", [1000, 2160])  # 8 and 16 columns per thread; 2160: 4 delay rows per CTA
def test_cylindrical_binning_wide_rows(nc):
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt = 16
    edges = [1.0, 3.0, 5.0]
    v = synth.sky_visibilities(nt, nc, seed=17)
    plan = bs.Plan(nt, nc, edges, precision=1)
    plan.grid_load(torch.from_numpy(v[None]).cuda())
    plan.mabs(accumulate=True)
    b3 = torch.empty((1, plan.n_closable, nc, nc), dtype=torch.float64, device="cuda")
    plan.bs3d_closable(b3)
    kpar = mo.kpar_axis(nc)
    ke = np.linspace(-0.7 * kpar.max(), 0.95 * kpar.max(), 17)
    sums, cnt = plan.bs_cylindrical(b3, kpar, ke)
    torch.cuda.synchronize()
    b3h = b3.cpu().numpy()
    q = mo.axis_bins(kpar, ke)
    n = len(ke) - 1
    na = np.bincount(q[q >= 0], minlength=n)
    np.testing.assert_array_equal(cnt.cpu().numpy(), np.outer(na, na))
    # sums by separable bin sums (row-bin x column-bin indicator matrices)
    ind = np.zeros((n, nc))
    ind[q[q >= 0], np.flatnonzero(q >= 0)] = 1.0
    want = np.einsum("qa,pab,rb->pqr", ind, b3h[0], ind)
    scale = np.abs(b3h).max() * np.maximum(cnt.cpu().numpy(), 1)
    assert np.all(np.abs(sums.cpu().numpy()[0] - want) <= 1e-12 * scale)
    plan.close()


@pytest.mark.parametrize("batch,lmax,nc", [(2, 4, 24), (1, 2, 23), (5, 3, 16)])
def test_multipoles_on_estimated_bispectrum(batch, lmax, nc):
    """bs_bs_multipoles on the GPU's own closable 3D bispectrum: counts and
    sums inside the oracle's interval; the odd l, which the point symmetry of
    the real part of a Hermitian 3D bispectrum cancels, vanish to rounding;
    one and several launches over realisations."""
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt, r, rp, dnu = 64, 900.0, 1.2, 0.16
    edges = synth.edges_log(8, 1.5, 31.0)
    v = np.stack([synth.sky_visibilities(nt, nc, seed=400 + s) for s in range(batch)])
    plan = bs.Plan(nt, nc, edges, precision=1, batch=batch, r=r, rprime=rp, dnu_c=dnu,
                   multires=True)
    plan.grid_load(torch.from_numpy(v).cuda())
    plan.mabs(accumulate=True)
    tri, _ = plan.counts()
    ncl = plan.n_closable
    b3 = torch.empty((batch, ncl, nc, nc), dtype=torch.float64, device="cuda")
    plan.bs3d_closable(b3)
    kperp = 2 * np.pi * plan.ring_umean() / r
    kpar = mo.kpar_axis(nc, rp, dnu)
    k1e = np.geomspace(0.5 * kperp.min(), 1.2 * np.sqrt(kperp.max() ** 2 + kpar.max() ** 2), 13)
    sums, cnt = plan.bs_multipoles(b3, kperp, kpar, k1e, 5, 5, lmax=lmax)
    torch.cuda.synchronize()
    b3h = b3.cpu().numpy()
    trips = _planes_trips(tri, len(edges) - 1)
    _, c_o = mo.bs_multipoles(b3h, trips, kperp, kpar, k1e, 5, 5, lmax)
    iv = mo.multipole_interval(b3h, trips, kperp, kpar, k1e, 5, 5, lmax, REL_K, REL_S)
    c = cnt.cpu().numpy()
    s = sums.cpu().numpy()
    assert s.shape == (batch, lmax + 1, 12, 5, 5)
    scale = np.abs(b3h).max() * 9 * np.maximum(iv["c_hi"], 1)
    _check_interval(c, s, iv, c_o, 1e-12 * scale)
    # l = 0 is the monopole over the same (paired) samples
    if nc % 2:
        s_m, c_m = plan.bs_monopole(b3, kperp, kpar, k1e, 5, 5)
        np.testing.assert_array_equal(c, c_m.cpu().numpy())
        np.testing.assert_allclose(s[:, 0], s_m.cpu().numpy(), rtol=1e-12,
                                   atol=1e-13 * scale.max())
    if lmax >= 1:
        # odd l of the point-symmetric part cancel; what is left comes from the
        # antisymmetric part A of the computed planes, |odd l| <= (2l+1) max|A| count
        lo = nc % 2 == 0
        refl = np.r_[0, nc - np.arange(1, nc)] if lo else nc - 1 - np.arange(nc)
        A = 0.5 * (b3h - b3h[:, :, refl][:, :, :, refl])[:, :, lo:, lo:]
        a_max = np.abs(A).max()
        odd = np.abs(s[:, 1::2]).max()
        even = np.abs(s[:, 0::2]).max()
        print(f"max |odd l| / max |even l| = {odd / even:.2e}; "
              f"max |A| / max |B| = {a_max / np.abs(b3h).max():.2e}")
        bound = (2 * lmax + 1) * a_max * c + 1e-12 * scale
        assert np.all(np.abs(s[:, 1::2]) <= bound[None, None])
        assert odd < 1e-5 * even
    plan.close()


def test_multipoles_argument_errors():
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt, nc = 32, 8
    edges = synth.edges_linear(4, 11)
    plan = bs.Plan(nt, nc, edges, precision=1)
    plan.grid_load(torch.from_numpy(synth.sky_visibilities(nt, nc, seed=5)[None]).cuda())
    plan.mabs()
    plan.counts()
    b3 = torch.zeros((1, plan.n_closable, nc, nc), dtype=torch.float64, device="cuda")
    kperp = 2 * np.pi * plan.ring_umean()
    kpar = mo.kpar_axis(nc)
    with pytest.raises(bs.BsError):
        plan.bs_multipoles(b3, kperp, kpar, [0.1, 1.0, 10.0], lmax=5)
    with pytest.raises(bs.BsError):
        plan.bs_multipoles(b3, kperp, kpar, [1.0, 0.1], lmax=2)
    plan.close()


def test_binnings_of_a_general_plan():
    """General (non-Hermitian) input, two realisations: the complex closable
    3D bispectrum binned by the monopole, the m = 0 multipoles and the
    (k_par1, k_par2) grid.  The binnings are linear, so the real and the
    imaginary part of every complex sum must pass the oracle checks that real
    values pass, with the same counts."""
    torch = _torch()
    import paper_2506_10526_gb300 as bs
    nt, nc, r, rp, dnu = 48, 24, 900.0, 1.2, 0.16
    edges = synth.edges_log(6, 1.5, 23.0)
    g = synth.rng(611)
    v = (g.standard_normal((2, nc, nt, nt)) + 1j * g.standard_normal((2, nc, nt, nt)))
    plan = bs.Plan(nt, nc, edges, precision=1, batch=2, r=r, rprime=rp, dnu_c=dnu,
                   multires=True, general=True)
    plan.grid_load(torch.from_numpy(v.astype(np.complex64)).cuda())
    plan.mabs(accumulate=True)
    tri, _ = plan.counts()
    b3 = torch.empty((2, plan.n_closable, nc, nc), dtype=torch.complex128, device="cuda")
    plan.bs3d_closable(b3)
    kperp = 2 * np.pi * plan.ring_umean() / r
    kpar = mo.kpar_axis(nc, rp, dnu)
    k1e = np.geomspace(0.5 * kperp.min(), 1.2 * np.sqrt(kperp.max() ** 2 + kpar.max() ** 2), 13)
    ke = np.linspace(-0.8 * kpar.max(), 0.8 * kpar.max(), 11)
    sums, cnt = plan.bs_monopole(b3, kperp, kpar, k1e, 5, 5)
    msums, mcnt = plan.bs_multipoles(b3, kperp, kpar, k1e, 5, 5, lmax=2)
    csums, ccnt = plan.bs_cylindrical(b3, kpar, ke)
    torch.cuda.synchronize()
    b3h = b3.cpu().numpy()
    assert np.abs(b3h.imag).max() > 0.1 * np.abs(b3h.real).max()  # really complex
    s, c = sums.cpu().numpy(), cnt.cpu().numpy()
    ms, mc = msums.cpu().numpy(), mcnt.cpu().numpy()
    cs, cc = csums.cpu().numpy(), ccnt.cpu().numpy()
    assert s.dtype == ms.dtype == cs.dtype == np.complex128
    assert s.shape == (2, 12, 5, 5) and ms.shape == (2, 3, 12, 5, 5)
    trips = _planes_trips(tri, len(edges) - 1)
    for part in (np.real, np.imag):
        x = np.ascontiguousarray(part(b3h))
        _, c_o = mo.bs_monopole(x, trips, kperp, kpar, k1e, 5, 5)
        iv = mo.monopole_interval(x, trips, kperp, kpar, k1e, 5, 5, REL_K, REL_S)
        _check_interval(c, part(s), iv, c_o, 1e-12 * np.abs(x).max() * np.maximum(iv["c_hi"], 1))
        _, cm_o = mo.bs_multipoles(x, trips, kperp, kpar, k1e, 5, 5, 2)
        ivm = mo.multipole_interval(x, trips, kperp, kpar, k1e, 5, 5, 2, REL_K, REL_S)
        scale = np.abs(x).max() * 9 * np.maximum(ivm["c_hi"], 1)
        _check_interval(mc, part(ms), ivm, cm_o, 1e-12 * scale)
        s_o, cc_o = mo.bs_cylindrical(x, kpar, ke)
        np.testing.assert_array_equal(cc, cc_o)
        assert np.all(np.abs(part(cs) - s_o) <= 1e-12 * np.abs(x).max() * np.maximum(cc_o, 1))
    plan.close()
