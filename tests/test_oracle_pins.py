"""Pins for the FP64 oracle: each check ties an oracle function to something
other than itself (a hand-worked example, brute force, a closed form, an
invariant of the estimator, or the analytic bispectrum of the test field).

Estimator: arXiv:2506.10526 Sec. 3.2, Eq. (estimator_t); collapse and fold:
Sec. 3.2 and Sec. 5 (Fig. Nv); delay transform: Eq. (dft); test field:
Eq. (mb1), Eq. (bsana)."""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hermitian_random(nc, nt, seed):
    """Random complex grid with V(-U) = conj V(U) on the binnable cells."""
    r = synth.rng(seed)
    a = r.standard_normal((nc, nt, nt)) + 1j * r.standard_normal((nc, nt, nt))
    out = np.zeros_like(a)
    h = nt // 2
    for iv in range(1, nt):
        for iu in range(1, nt):
            jv, ju = nt - iv, nt - iu  # -(v) + h = nt - iv when iv = v + h
            out[:, iv, iu] = 0.5 * (a[:, iv, iu] + np.conj(a[:, jv, ju]))
    out[:, 0, :] = a[:, 0, :]
    out[:, :, 0] = a[:, :, 0]
    return out


def _brute_force(vis, edges, ngrid=None, chan_flags=None):
    """O(N_cells^3) brute force: every ordered triple of binned cells is tested
    for closure U1 + U2 + U3 = 0; no pair lookup is used."""
    nc, nt, _ = vis.shape
    lab = oracle.ring_labels(nt, edges)
    w, wn = oracle.weights(nc, nt, ngrid, chan_flags)
    x = vis * w
    iv, iu = np.nonzero(lab >= 0)
    u = iu - nt // 2
    v = iv - nt // 2
    r = lab[iv, iu]
    close = ((u[:, None, None] + u[None, :, None] + u[None, None, :]) == 0) & \
            ((v[:, None, None] + v[None, :, None] + v[None, None, :]) == 0)
    a, b, c = np.nonzero(close)
    nb = len(edges) - 1
    trip = oracle.ring_triples(nb)
    index = {t: k for k, t in enumerate(trip)}
    num = np.zeros((len(trip), nc, nc, nc), complex)
    den = np.zeros((len(trip), nc, nc, nc))
    cnt = np.zeros(len(trip), np.int64)
    xc = x[:, iv, iu]  # [nc, cell]
    yc = wn[:, iv, iu]
    for p, q, s in zip(a, b, c):
        key = (r[p], r[q], r[s])
        if key not in index:
            continue
        k = index[key]
        cnt[k] += 1
        num[k] += np.einsum("i,j,l->ijl", xc[:, p], xc[:, q], xc[:, s])
        den[k] += np.einsum("i,j,l->ijl", yc[:, p], yc[:, q], yc[:, s])
    return num, den, cnt


def test_three_mode_golden():
    """Hand-derived values (tests/golden/three_mode.txt)."""
    kv = {}
    for line in open(os.path.join(GOLDEN, "three_mode.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, *vals = line.split()
            kv[k] = [float(x) for x in vals]
    nt = int(kv["nt"][0])
    vis = np.zeros((1, nt, nt), complex)
    for key, val in (("U_a", "a"), ("U_b", "b"), ("U_c", "c")):
        u, v = (int(t) for t in kv[key])
        z = complex(*kv[val])
        vis[0, v + nt // 2, u + nt // 2] = z
        vis[0, -v + nt // 2, -u + nt // 2] = np.conj(z)
    res = oracle.mabs_full(vis, kv["edges"])
    idx = {t: k for k, t in enumerate(res["triples"])}
    assert res["T"][idx[(0, 0, 1)]] == int(kv["T_001"][0])
    assert res["T"][idx[(0, 0, 0)]] == int(kv["T_000"][0])
    assert res["B"][idx[(0, 0, 1)]].ravel()[0] == pytest.approx(kv["B_001"][0], abs=1e-15)
    assert res["B"][idx[(0, 0, 0)]].ravel()[0] == pytest.approx(kv["B_000"][0], abs=1e-15)


@pytest.mark.parametrize("nt,nc,edges,seed", [(8, 3, [1.0, 2.0, 3.0, 4.0], 11),
                                               (16, 2, [1.0, 3.0, 5.0, 8.0], 12)])
def test_enumeration_matches_brute_force(nt, nc, edges, seed):
    """Pair enumeration == O(N^3) closure test, with empty cells, non-unit
    sampling counts and one flagged channel."""
    vis = _hermitian_random(nc, nt, seed)
    r = synth.rng(seed + 100)
    ngrid = r.integers(0, 4, size=(nc, nt, nt)).astype(float)
    flags = np.zeros(nc, np.uint8)
    flags[-1] = 1
    res = oracle.mabs_full(vis, edges, ngrid=ngrid, chan_flags=flags)
    num, den, _ = _brute_force(vis, edges, ngrid=ngrid, chan_flags=flags)
    scale = np.abs(num).max()
    np.testing.assert_allclose(res["num"], num, atol=1e-12 * scale, rtol=0)
    np.testing.assert_allclose(res["den"], den, atol=1e-12 * np.abs(den).max(), rtol=0)
    # geometric counts (no occupancy) against brute force on an unweighted grid
    _, _, cnt = _brute_force(vis, edges)
    np.testing.assert_array_equal(res["T"], cnt)


def test_enumeration_matches_brute_force_general_input():
    """Visibilities with no symmetry at all (V(-U) unrelated to V(U)*) and an
    asymmetric sampling grid: complex numerators, pair enumeration against the
    O(N^3) closure test; Hermitian input gives real numerators (the imaginary
    parts here are not small)."""
    nt, nc, edges = 12, 3, [1.0, 2.5, 4.0, 5.5]
    r = synth.rng(31)
    vis = r.standard_normal((nc, nt, nt)) + 1j * r.standard_normal((nc, nt, nt))
    ngrid = r.integers(0, 3, size=(nt, nt)).astype(float)
    res = oracle.mabs_full(vis, edges, ngrid=ngrid)
    num, den, _ = _brute_force(vis, edges, ngrid=ngrid)
    scale = np.abs(num).max()
    np.testing.assert_allclose(res["num"], num, atol=1e-12 * scale, rtol=0)
    np.testing.assert_allclose(res["den"], den, atol=1e-12 * np.abs(den).max(), rtol=0)
    assert np.abs(res["num"].imag).max() > 0.1 * scale


def test_counts_invariants():
    """T(i,j,l) is invariant under permutations of (i, j, l); summing over l
    gives the number of ordered pairs (g1 in a_i, g2 in a_j) whose closing
    point -g1-g2 is binned; counts from the separate count routine agree
    with the counts of the enumeration."""
    nt = 32
    edges = synth.edges_linear(5, 16)
    T = oracle.counts(nt, edges)
    for perm in [(0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]:
        np.testing.assert_array_equal(T, np.transpose(T, perm))
    lab = oracle.ring_labels(nt, edges)
    iv, iu = np.nonzero(lab >= 0)
    u, v, rr = iu - nt // 2, iv - nt // 2, lab[iv, iu]
    u3 = -(u[:, None] + u[None, :])
    v3 = -(v[:, None] + v[None, :])
    inside = (np.abs(u3) < nt // 2) & (np.abs(v3) < nt // 2)
    closes = np.zeros_like(inside)
    closes[inside] = lab[v3[inside] + nt // 2, u3[inside] + nt // 2] >= 0
    nb = len(edges) - 1
    for i in range(nb):
        for j in range(nb):
            want = closes[np.ix_(rr == i, rr == j)].sum()
            assert T[i, j].sum() == want
    vis = np.ones((1, nt, nt), complex)
    res = oracle.mabs_full(vis, edges)
    for k, (i, j, l) in enumerate(res["triples"]):
        assert res["T"][k] == T[i, j, l]


def test_counts_small_rings_by_hand():
    """Rings with four cells each: ring 0 = the unit axis cells (|U|^2 = 1),
    ring 1 = the diagonal cells (+-1, +-1) (|U|^2 = 2), ring 2 = the axis
    cells at radius 2 (|U|^2 = 4).  Counted by hand:
      T(0,0,2) = 4  (g + g = 2g),   T(0,0,1) = 8  (perpendicular unit pairs),
      T(0,1,0) = 8  (unit + diagonal = unit),  T(1,1,2) = 8  ((1,1)+(1,-1)),
      T(0,0,0) = T(1,1,1) = T(2,2,2) = 0."""
    edges = [1.0, 1.1, 2.0, 2.1]
    T = oracle.counts(16, edges)
    for (i, j, l), n in {(0, 0, 2): 4, (0, 0, 1): 8, (0, 1, 0): 8, (1, 1, 2): 8,
                         (0, 0, 0): 0, (1, 1, 1): 0, (2, 2, 2): 0}.items():
        for perm in {(i, j, l), (i, l, j), (j, i, l), (j, l, i), (l, i, j), (l, j, i)}:
            assert T[perm] == n, (perm, T[perm], n)


def _cfg_small(seed=5, nt=16, nc=4):
    vis = synth.sky_visibilities(nt, nc, seed, dtype=np.complex128)
    return vis, [1.0, 3.0, 5.0, 7.5]


def test_constant_fields():
    """V == 1 gives B = 1/A in every valid bin; V = c(nu) real gives
    c(nu1) c(nu2) c(nu3) / A; a flagged channel gives NaN."""
    nt, nc = 16, 4
    edges = [1.0, 3.0, 5.0, 7.5]
    A = 2.5
    res = oracle.mabs_full(np.ones((nc, nt, nt), complex), edges, norm_A=A)
    B = res["B"]
    ok = res["T"] > 0
    np.testing.assert_allclose(B[ok], 1.0 / A, rtol=1e-13)
    assert np.all(np.isnan(B[~ok]))
    c = np.array([1.0, -2.0, 0.5, 3.0])
    flags = np.array([0, 0, 1, 0], np.uint8)
    res = oracle.mabs_full(np.ones((nc, nt, nt)) * c[:, None, None], edges, chan_flags=flags)
    want = np.einsum("i,j,l->ijl", c, c, c)
    for k in np.nonzero(res["T"] > 0)[0]:
        got = res["B"][k]
        valid = np.einsum("i,j,l->ijl", 1 - flags, 1 - flags, 1 - flags).astype(bool)
        np.testing.assert_allclose(got[valid], want[valid], rtol=1e-12)
        assert np.all(np.isnan(got[~valid]))


def test_scaling_translation_rotation_reflection():
    """B(alpha V) = alpha^3 B(V); a phase gradient exp(-2 pi i U.s) leaves B
    unchanged (closure phase is 1); a 90-degree rotation or a reflection of
    the uv plane leaves B unchanged (rings are isotropic)."""
    vis, edges = _cfg_small()
    nc, nt, _ = vis.shape
    base = oracle.mabs_full(vis, edges)["B"]
    ok = ~np.isnan(base)
    scale = np.nanmax(np.abs(base))
    alpha = 1.7 - 0.4j
    np.testing.assert_allclose(oracle.mabs_full(alpha * vis, edges)["B"][ok],
                               alpha**3 * base[ok], atol=1e-12 * scale * abs(alpha) ** 3)
    u = np.arange(nt) - nt // 2
    uu, vv = np.meshgrid(u, u, indexing="xy")
    s = (0.37, -1.21)
    ph = np.exp(-2j * np.pi * (uu * s[0] + vv * s[1]) / nt)
    np.testing.assert_allclose(oracle.mabs_full(vis * ph, edges)["B"][ok], base[ok],
                               atol=1e-12 * scale)
    # rotation (u, v) -> (-v, u): V'(u, v) = V(v, -u)
    rot = np.zeros_like(vis)
    ref = np.zeros_like(vis)
    h = nt // 2
    for iv in range(1, nt):
        for iu in range(1, nt):
            uq, vq = iu - h, iv - h
            rot[:, iv, iu] = vis[:, -uq + h, vq + h]
            ref[:, iv, iu] = vis[:, vq + h, -uq + h]
    np.testing.assert_allclose(oracle.mabs_full(rot, edges)["B"][ok], base[ok], atol=1e-12 * scale)
    np.testing.assert_allclose(oracle.mabs_full(ref, edges)["B"][ok], base[ok], atol=1e-12 * scale)


def test_channel_permutation_and_hermitian_reality():
    """Permuting the channels permutes the cube; Hermitian input gives a real
    estimator (imaginary part at rounding level)."""
    vis, edges = _cfg_small(nc=5)
    perm = np.array([3, 0, 4, 1, 2])
    a = oracle.mabs_full(vis, edges)["B"]
    b = oracle.mabs_full(vis[perm], edges)["B"]
    ok = ~np.isnan(a)
    np.testing.assert_allclose(b[:, :, :, :][ok[:, perm][:, :, perm][:, :, :, perm]],
                               a[:, perm][:, :, perm][:, :, :, perm][ok[:, perm][:, :, perm][:, :, :, perm]],
                               rtol=1e-12, atol=1e-12 * np.nanmax(np.abs(a)))
    assert np.nanmax(np.abs(a.imag)) <= 1e-12 * np.nanmax(np.abs(a.real))


def test_points_match_full_cube():
    vis, edges = _cfg_small(nc=3)
    res = oracle.mabs_full(vis, edges, chan_flags=[0, 1, 0])
    pts = []
    want = []
    for k, (i, j, l) in enumerate(res["triples"]):
        for n1, n2, n3 in [(0, 2, 1), (2, 2, 0), (1, 0, 2)]:
            pts.append((i, j, l, n1, n2, n3))
            want.append(res["B"][k, n1, n2, n3])
    got, _ = oracle.mabs_points(vis, edges, pts, chan_flags=[0, 1, 0])
    want = np.array(want)
    np.testing.assert_array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    np.testing.assert_allclose(got[ok], want[ok], rtol=1e-12, atol=1e-13 * np.abs(want[ok]).max())


def test_n_nu_closed_form_and_flags():
    """Unflagged: N_nu(d1, d2) = max(0, nc - (max(0,d1,d2) - min(0,d1,d2))),
    N_nu(0,0) = nc (Sec. 5, Fig. Nv); zero exactly where the spread of the
    three channels reaches nc.  With the coarse-band flags, N_nu has no zero
    inside the square |d| <= nc/2 (Sec. 5) except next to its two corners,
    where even the unflagged sampling has fewer than one coarse band of
    channel triples (the corners themselves are unsampled without flags)."""
    for nc in (1, 7, 16):
        N = oracle.n_nu(np.ones(nc, bool))
        d = np.arange(-(nc - 1), nc)
        D1, D2 = np.meshgrid(d, d, indexing="ij")
        spread = np.maximum(0, np.maximum(D1, D2)) - np.minimum(0, np.minimum(D1, D2))
        np.testing.assert_array_equal(N, np.maximum(0, nc - spread))
        assert N[nc - 1, nc - 1] == nc
        F = oracle.fold_plane(N)
        assert F[nc - 1, nc - 1] == nc
        if nc > 1:
            assert F[nc, nc - 1] == 2 * N[nc, nc - 1]
    for nc in (16, 64, 96):
        h = nc // 2
        sq = slice(nc - 1 - h, nc + h)
        full = oracle.fold_plane(oracle.n_nu(np.ones(nc, bool)))[sq, sq]
        # unflagged: inside the square only the two corners (-h, h), (h, -h),
        # whose channel spread equals nc, are unsampled
        zeros = np.argwhere(full == 0) - h
        assert sorted(map(tuple, zeros)) == [(-h, h), (h, -h)]
        valid = synth.flag_mask_coarse_band(nc) == 0
        flagged = oracle.fold_plane(oracle.n_nu(valid))[sq, sq]
        # flags open no hole where at least one coarse band of triples exists
        assert flagged[full >= min(32, nc // 2)].min() > 0
        assert flagged.sum() < full.sum()


def test_collapse_fold_ratio_identity():
    """With every cell filled and channel-only flags, every valid channel
    triple of a ring triple has the same denominator, so the mean of ratios
    equals (sum of numerators) / (T * N_nu); the folded plane is point
    symmetric; the C collapsed-plane points agree with the cube."""
    vis, edges = _cfg_small(nc=6)
    flags = np.array([0, 1, 0, 0, 0, 1], np.uint8)
    res = oracle.mabs_full(vis, edges, chan_flags=flags)
    bbar, cnt = oracle.collapse_fold(res["B"])
    nc = 6
    valid = flags == 0
    nn = oracle.fold_plane(oracle.n_nu(valid))
    for k in np.nonzero(res["T"] > 0)[0]:
        s = np.zeros((2 * nc - 1, 2 * nc - 1), complex)
        for n1 in range(nc):
            for n2 in range(nc):
                for n3 in range(nc):
                    if valid[n1] and valid[n2] and valid[n3]:
                        s[n1 - n3 + nc - 1, n2 - n3 + nc - 1] += res["num"][k, n1, n2, n3]
        want = oracle.fold_plane(s) / (res["T"][k] * np.where(nn > 0, nn, 1))
        ok = nn > 0
        np.testing.assert_allclose(bbar[k][ok], want[ok], rtol=1e-12,
                                   atol=1e-12 * np.abs(want).max())
        assert np.all(np.isnan(bbar[k][~ok]))
        np.testing.assert_array_equal(cnt[k], nn)
    np.testing.assert_allclose(bbar, bbar[:, ::-1, ::-1], rtol=1e-13, atol=0, equal_nan=True)
    k = int(np.nonzero(res["T"] > 0)[0][-1])
    i, j, l = res["triples"][k]
    pts = [(i, j, l, d1, d2) for d1, d2 in [(0, 0), (2, -1), (-3, 4), (5, 5), (1, 3)]]
    got, c2 = oracle.delta_points(vis, edges, pts, chan_flags=flags)
    for p, g, cc in zip(pts, got, c2):
        w = bbar[k, p[3] + nc - 1, p[4] + nc - 1]
        assert cc == cnt[k, p[3] + nc - 1, p[4] + nc - 1]
        if np.isnan(w):
            assert np.isnan(g)
        else:
            assert g == pytest.approx(w, rel=1e-12, abs=1e-12 * np.nanmax(np.abs(bbar[k])))


def test_collapse_ratio_of_sums_for_per_channel_sampling():
    """The ratio-of-sums collapse (per-channel sampling): equal to the mean of
    the estimates with one sampling grid; a constant field c gives c^3 / A at
    every sampled separation whatever the per-channel occupancy; a field c(nu)
    gives the mean of c1 c2 c3 weighted by the closed-triangle counts of the
    occupied cells (those counts from the O(N^3) brute force)."""
    nt, nc = 16, 4
    vis, edges = _cfg_small(nt=nt, nc=nc)
    res = oracle.mabs_full(vis, edges)
    r = oracle.collapse_fold_ratio(res["num"], res["den"])
    bbar, _ = oracle.collapse_fold(res["B"])
    keep = res["T"] > 0
    ok = ~np.isnan(bbar[keep])
    np.testing.assert_allclose(r[keep][ok], bbar[keep][ok], rtol=1e-12,
                               atol=1e-12 * np.nanmax(np.abs(bbar[keep])))
    # per-channel occupancy, symmetric in U for each channel
    g = synth.rng(41)
    occ = g.integers(0, 2, size=(nc, nt, nt)).astype(float)
    occ[:, 1:, 1:] = np.maximum(occ[:, 1:, 1:], occ[:, 1:, 1:][:, ::-1, ::-1])
    c = np.array([1.5, -0.5, 2.0, 0.75])
    for field in (np.full(nc, 1.3), c):
        v = field[:, None, None] * occ  # N_g visibilities of value c(nu) per cell
        rr = oracle.mabs_full(v.astype(complex), edges, ngrid=occ, norm_A=2.0)
        got = oracle.collapse_fold_ratio(rr["num"], rr["den"], norm_A=2.0)
        _, den, _ = _brute_force(v.astype(complex), edges, ngrid=occ)
        w = np.einsum("i,j,l->ijl", field, field, field)
        for k in np.flatnonzero(rr["T"] > 0):
            for d1 in range(-(nc - 1), nc):
                for d2 in range(-(nc - 1), nc):
                    num_w = den_w = 0.0
                    for sgn in ((1,) if d1 == d2 == 0 else (1, -1)):
                        for n3 in range(nc):
                            n1, n2 = n3 + sgn * d1, n3 + sgn * d2
                            if 0 <= n1 < nc and 0 <= n2 < nc:
                                num_w += w[n1, n2, n3] * den[k, n1, n2, n3]
                                den_w += den[k, n1, n2, n3]
                    x = got[k, d1 + nc - 1, d2 + nc - 1]
                    if den_w == 0:
                        assert np.isnan(x)
                    else:
                        assert x.real == pytest.approx(num_w / den_w / 2.0, rel=1e-12)
        if np.all(field == field[0]):
            fin = np.isfinite(got.real)
            np.testing.assert_allclose(got.real[fin], field[0] ** 3 / 2.0, rtol=1e-12)


def test_delta_points_rectangular_block():
    """The collapsed-plane points of a rectangular channel block (nu1, nu2 in
    one range, nu3 in another) against a brute-force mean over the full
    cube's channel triples inside the block."""
    vis, edges = _cfg_small(nc=7)
    res = oracle.mabs_full(vis, edges)
    nc = 7
    blk = (1, 4, 0, 3, 2, 7)
    k = int(np.nonzero(res["T"] > 0)[0][-1])
    i, j, l = res["triples"][k]
    pts = [(i, j, l, d1, d2) for d1, d2 in [(0, 0), (1, -1), (-2, -3), (-1, 0), (3, 3)]]
    got, cnt = oracle.delta_points(vis, edges, pts, block=blk)
    for p, g, c in zip(pts, got, cnt):
        vals = []
        for sgn in ((1,) if p[3] == p[4] == 0 else (1, -1)):
            d1, d2 = sgn * p[3], sgn * p[4]
            for n3 in range(blk[4], blk[5]):
                n1, n2 = n3 + d1, n3 + d2
                if blk[0] <= n1 < blk[1] and blk[2] <= n2 < blk[3]:
                    vals.append(res["B"][k, n1, n2, n3])
        assert c == len(vals)
        if vals:
            assert g == pytest.approx(np.mean(vals), rel=1e-12, abs=1e-12 * np.abs(vals).max())
        else:
            assert np.isnan(g)


def _placed(plane, nc, lo):
    """Put the separations n = lo .. lo + nc - 1 of a centred plane at
    indices n mod nc (one full period of the nc-periodic DFT kernel)."""
    n = np.arange(lo, lo + nc)
    sub = plane[n + nc - 1][:, n + nc - 1]
    out = np.zeros((nc, nc), complex)
    out[np.ix_(n % nc, n % nc)] = sub
    return out


@pytest.mark.parametrize("nc", [8, 16, 7])
def test_delay_dft_closed_forms(nc):
    """Eq. (dft), half-open range n, m in [-nc/2, nc/2) (one period), on planes
    with known transforms: a constant plane (a single spike), a separable
    cosine (four spikes), and agreement with numpy's FFT of the same nc x nc
    separations (with Parseval).  Output index a + nc//2 holds k_par index a."""
    h = nc // 2
    d = np.arange(-(nc - 1), nc)
    D1, D2 = np.meshgrid(d, d, indexing="ij")
    const = np.ones((2 * nc - 1, 2 * nc - 1))
    out = oracle.delay_dft(const, nc)
    want = np.zeros((nc, nc))
    want[h, h] = nc * nc
    np.testing.assert_allclose(out, want, atol=1e-10 * nc * nc)
    p, q = 2, 3
    cosp = np.cos(2 * np.pi * p * D1 / nc) * np.cos(2 * np.pi * q * D2 / nc)
    out = oracle.delay_dft(cosp, nc, r=1.3, rprime=0.7, dnu_c=0.04)
    scale = (1.3**2 * 0.7 * 0.04) ** 2
    spikes = np.abs(out) > 1e-6 * np.abs(out).max()
    assert spikes.sum() == 4
    for aa in (p, -p):
        for bb in (q, -q):
            assert spikes[aa + h, bb + h]
            assert out[aa + h, bb + h].real == pytest.approx(scale * nc * nc / 4, rel=1e-12)
    rnd = synth.rng(nc).standard_normal((2 * nc - 1, 2 * nc - 1))
    rnd = rnd + rnd[::-1, ::-1]  # point symmetric, as a folded plane is
    out = oracle.delay_dft(rnd, nc)
    per = _placed(rnd, nc, -h)
    np.testing.assert_allclose(out, np.roll(np.fft.fft2(per), (h, h), axis=(0, 1)),
                               atol=1e-10 * np.abs(out).max())
    assert np.sum(np.abs(out) ** 2) == pytest.approx(nc * nc * np.sum(np.abs(per) ** 2), rel=1e-12)
    # real part = mean of the two half-open ranges [-h, h) and (-h, h]
    other = np.roll(np.fft.fft2(_placed(rnd, nc, -h + 1 if nc % 2 == 0 else -h)), (h, h), axis=(0, 1))
    np.testing.assert_allclose(out.real, 0.5 * (out + other).real, atol=1e-10 * np.abs(out).max())
    if nc % 2 == 1:  # the half-open range is symmetric: the output is real
        assert np.abs(out.imag).max() <= 1e-10 * np.abs(out.real).max()


@pytest.mark.parametrize("nc", [8, 7])
def test_delay_dft_inclusive_variant_differs_by_the_end_terms(nc):
    """The printed limits -nc/2 ... nc/2 read literally (both ends) add, for
    even nc, the row n = nc/2 and the column m = nc/2 to the half-open sum;
    for odd nc the two readings are the same sum."""
    h = nc // 2
    rnd = synth.rng(100 + nc).standard_normal((2 * nc - 1, 2 * nc - 1))
    half = oracle.delay_dft(rnd, nc)
    incl = oracle.delay_dft(rnd, nc, variant="inclusive")
    if nc % 2 == 1:
        np.testing.assert_allclose(incl, half, atol=1e-12 * np.abs(half).max())
        return
    a = np.arange(-h, -h + nc)
    ninc = np.arange(-h, h + 1)
    extra = np.zeros((nc, nc), complex)
    for n in ninc:
        for m in ninc:
            if n == h or m == h:
                extra += rnd[n + nc - 1, m + nc - 1] * np.exp(
                    -2j * np.pi * (np.add.outer(n * a, m * a)) / nc)
    np.testing.assert_allclose(incl - half, extra, atol=1e-10 * np.abs(incl).max())
    assert np.abs(extra).max() > 1e-3 * np.abs(half).max()  # the difference is visible


def _ensemble_z(nreal=400, f_ng=1.0, predict=None):
    """|z| of the ensemble-mean estimator against a prediction, per
    (ring triple, separation) bin, for the Eq. (mb1) field on a 12^2 x 6 box."""
    nt, nc, sigma = 12, 6, 0.5
    edges = [1.0, 2.5, 4.0, 5.5]
    p = synth.grf_power(nt, nc, -2.0, sigma)
    cubes = []
    for s in range(nreal):
        vis = synth.sky_visibilities(nt, nc, 5000 + s, f_ng=f_ng, sigma=sigma,
                                     dtype=np.complex128)
        res = oracle.mabs_full(vis, edges)
        cubes.append(res["B"].real)
    cubes = np.array(cubes)  # [nreal, ntrip, nc, nc, nc]
    trip = res["triples"]
    keep = [k for k in range(len(trip)) if res["T"][k] > 0]
    dpairs = [(0, 0), (1, 0), (0, 2), (1, -1), (2, 3), (-1, 2), (3, 0)]
    predict = predict or oracle.analytic_mabs
    pred = predict(nt, nc, edges, p, f_ng, [trip[k] for k in keep], dpairs)
    z = []
    for kk, k in enumerate(keep):
        for di, (d1, d2) in enumerate(dpairs):
            # collapse to (d1, d2): mean over the channel triples with that separation
            xs = [cubes[:, k, n3 + d1, n3 + d2, n3] for n3 in range(nc)
                  if 0 <= n3 + d1 < nc and 0 <= n3 + d2 < nc]
            x = np.mean(xs, axis=0)
            z.append((x.mean() - pred[kk, di].real) / (x.std(ddof=1) / np.sqrt(nreal)))
    return np.abs(np.array(z))


def test_analytic_bispectrum_ensemble():
    """Ensemble mean of Eq. (estimator_t), collapsed to (d1, d2), over 400
    seeded realisations of the Eq. (mb1) field (f_NG = 1, sigma = 0.5)
    agrees with the exact discrete bispectrum (tree term of Eq. bsana plus
    the f^3 loop term): every bin within 5 sigma/sqrt(N) (the Sec. 5 bound on
    Delta_sigma) and nearly all within 3 (Fig. mabs)."""
    z = _ensemble_z()
    assert z.max() < 5.0, z.max()
    assert np.mean(z < 3.0) >= 0.95


def test_analytic_pin_detects_planted_mistakes():
    """Planted mistakes in the oracle's prediction (on the CPU) fail the same
    comparison: dropping the loop term, dropping one tree term, or a factor 2."""
    def no_loop(nt, nc, edges, p, f_ng, triples, d_pairs):
        eps = 1e-9
        return oracle.analytic_mabs(nt, nc, edges, p, eps, triples, d_pairs) * (f_ng / eps)

    def double(*a):
        return 2.0 * oracle.analytic_mabs(*a)

    def missing_tree_term(nt, nc, edges, p, f_ng, triples, d_pairs):
        orig = oracle.box_bispectrum

        def bad(p_, f, k1, k2, ltab=None):
            shp = np.array(p_.shape)
            k1m, k2m = np.asarray(k1) % shp, np.asarray(k2) % shp
            k3m = (-k1m - k2m) % shp
            P1 = p_[k1m[..., 0], k1m[..., 1], k1m[..., 2]]
            P3 = p_[k3m[..., 0], k3m[..., 1], k3m[..., 2]]
            return orig(p_, f, k1, k2, ltab) - 2.0 * f * P3 * P1
        oracle.box_bispectrum = bad
        try:
            return oracle.analytic_mabs(nt, nc, edges, p, f_ng, triples, d_pairs)
        finally:
            oracle.box_bispectrum = orig

    for wrong in (no_loop, double, missing_tree_term):
        assert _ensemble_z(predict=wrong).max() > 8.0, wrong.__name__
