"""Pins of the monopole binning oracle (oracle/monopole.py) to the paper's
statements and to independent routes: the corners and edges of the (mu, t)
plane named in Section 5, explicit 3D vectors for Eq. (shape), a pure-Python
binning by linear search, the closed form of Eq. (bsana) for equilateral
triangles, and ring centres of hand-counted rings."""
import math

import numpy as np
import pytest

from oracle import monopole as mo


def _shape(k1, k2, k3):
    K1, mu, t = mo.triangle_shape(k1 * k1, k2 * k2, k3 * k3)
    return float(K1), float(mu), float(t)


def test_shape_corners_named_in_the_paper():
    # equilateral: upper-left corner of the (mu, t) plane
    assert _shape(1.0, 1.0, 1.0) == pytest.approx((1.0, 0.5, 1.0), abs=1e-15)
    # squeezed (k1 = k2, k3 -> 0): upper-right corner
    K1, mu, t = _shape(1.0, 1.0, 1e-7)
    assert (mu, t) == pytest.approx((1.0, 1.0), abs=1e-12)
    # stretched (k1 / 2 = k2 = k3): lower-right corner
    assert _shape(2.0, 1.0, 1.0)[1:] == pytest.approx((1.0, 0.5), abs=1e-15)
    # linear (collinear, k1 = k2 + k3): right boundary mu = 1
    assert _shape(1.0, 0.7, 0.3)[1] == pytest.approx(1.0, abs=1e-15)
    # L-isosceles (two larger sides equal): upper boundary t = 1
    assert _shape(1.0, 1.0, 0.6)[2] == 1.0
    # S-isosceles (two smaller sides equal): lower boundary 2 mu t = 1
    _, mu, t = _shape(1.0, 0.8, 0.8)
    assert 2 * mu * t == pytest.approx(1.0, abs=1e-15)
    # argument order does not matter
    assert _shape(0.6, 1.0, 0.9) == _shape(1.0, 0.9, 0.6)


def test_shape_against_explicit_vectors():
    """mu = -k1.k2 / (k1 k2) from explicit 3D vectors (two random vectors, the
    third closing the triangle) against the squared-length form."""
    r = np.random.default_rng(5)
    for _ in range(2000):
        a, b = r.normal(size=3), r.normal(size=3) * r.uniform(0.1, 3.0)
        vecs = sorted([a, b, -(a + b)], key=lambda v: -np.dot(v, v))
        k1, k2 = vecs[0], vecs[1]
        mu_v = -np.dot(k1, k2) / (np.linalg.norm(k1) * np.linalg.norm(k2))
        t_v = np.linalg.norm(k2) / np.linalg.norm(k1)
        K1, mu, t = mo.triangle_shape(*(np.dot(v, v) for v in (a, b, -(a + b))))
        assert mu == pytest.approx(mu_v, abs=1e-12)
        assert t == pytest.approx(t_v, abs=1e-13)
        assert K1 == pytest.approx(np.linalg.norm(k1), rel=1e-15)
        # the parameter range stated after Eq. (shape)
        assert 0.5 - 1e-12 <= mu <= 1 + 1e-12 and 0.5 - 1e-12 <= t <= 1
        assert 2 * mu * t >= 1 - 1e-12


def _brute_monopole(b3d, trips, kperp, kpar, k1_edges, n_mu, n_t):
    """Per-sample loops, bins found by linear search over their edges."""
    n_k1 = len(k1_edges) - 1
    batch, _, nc, _ = b3d.shape
    sums = np.zeros((batch, n_k1, n_mu, n_t))
    cnt = np.zeros((n_k1, n_mu, n_t), np.int64)
    tol = mo.SHAPE_TOL
    mu_e = [0.5 + 0.5 * q / n_mu for q in range(n_mu + 1)]
    t_e = [0.5 + 0.5 * q / n_t for q in range(n_t + 1)]
    for p, (i, j, l) in enumerate(trips):
        for ia in range(nc):
            for ib in range(nc):
                za, zb = kpar[ia], kpar[ib]
                sides = [math.sqrt(kperp[i] ** 2 + za ** 2), math.sqrt(kperp[j] ** 2 + zb ** 2),
                         math.sqrt(kperp[l] ** 2 + (za + zb) ** 2)]
                sides.sort(reverse=True)
                k1, k2, k3 = sides
                mu = (k1 * k1 + k2 * k2 - k3 * k3) / (2 * k1 * k2)
                t = k2 / k1
                if not (0.5 - tol <= mu <= 1 + tol and 0.5 - tol <= t <= 1 + tol):
                    continue
                mu, t = min(max(mu, 0.5), 1.0), min(max(t, 0.5), 1.0)
                qk = next((q for q in range(n_k1) if k1_edges[q] <= k1 < k1_edges[q + 1]), None)
                if qk is None:
                    continue
                qm = next(q for q in range(n_mu) if mu < mu_e[q + 1] or q == n_mu - 1)
                qt = next(q for q in range(n_t) if t < t_e[q + 1] or q == n_t - 1)
                cnt[qk, qm, qt] += 1
                sums[:, qk, qm, qt] += b3d[:, p, ia, ib]
    return sums, cnt


def test_monopole_binning_against_brute_force():
    r = np.random.default_rng(11)
    nb, nc = 4, 10
    kperp = np.sort(r.uniform(0.05, 0.3, nb))
    trips = [(0, 0, 0), (0, 1, 1), (0, 1, 2), (1, 2, 3), (2, 3, 3), (3, 3, 3)]
    kpar = mo.kpar_axis(nc, rprime=30.0, dnu_c=0.05)
    b3d = r.normal(size=(2, len(trips), nc, nc))
    edges = np.geomspace(0.04, 2.5, 7)
    s, c = mo.bs_monopole(b3d, trips, kperp, kpar, edges, 5, 5)
    s_b, c_b = _brute_monopole(b3d, trips, kperp, kpar, edges, 5, 5)
    # both decide bins in FP64 from the definition, by different routes
    np.testing.assert_array_equal(c, c_b)
    np.testing.assert_allclose(s, s_b, rtol=1e-12, atol=1e-12)
    assert 0 < c.sum() <= len(trips) * nc * nc


def test_bsana_closed_form_and_equilateral_bin():
    """Eq. (bsana) with P = k^-2 on an equilateral triangle is 6 f k^-4; a
    single equilateral sample (nc = 1: a = b = 0) lands in the first mu bin
    and the last t bin of the k1 bin holding k."""
    kap, f = 0.2, 0.7
    assert mo.bsana(kap ** 2, kap ** 2, kap ** 2, f, 1.0, -2.0) == pytest.approx(6 * f * kap ** -4,
                                                                              rel=1e-14)
    v = mo.bsana(0.3, 0.5, 0.7, f, 2.0, -2.0)
    assert v == pytest.approx(mo.bsana(0.7, 0.3, 0.5, f, 2.0, -2.0), rel=1e-15)
    edges = np.array([0.1, 0.15, 0.25, 0.4])
    s, c = mo.bs_monopole(None, [(0, 0, 0)], np.array([kap]), np.array([0.0]), edges, 5, 5,
                          model=(f, 1.0, -2.0))
    assert c.sum() == 1 and c[1, 0, 4] == 1
    assert s[0, 1, 0, 4] == pytest.approx(6 * f * kap ** -4, rel=1e-14)


def test_ring_mean_u_hand_counted_rings():
    nt = 16
    # [1, 1.2): the four cells at |U| = 1;  [1.4, 1.5): four at sqrt 2;
    # [1.9, 2.1): four at 2;  [2.2, 2.3): the eight at sqrt 5
    u = mo.ring_mean_u(nt, [1.0, 1.2, 1.4, 1.5, 1.9, 2.1, 2.2, 2.3])
    assert u[0] == 1.0
    assert u[2] == pytest.approx(math.sqrt(2), rel=1e-15)
    assert u[4] == 2.0
    assert u[6] == pytest.approx(math.sqrt(5), rel=1e-15)
    # empty ring: the mid point of its edges
    assert u[1] == pytest.approx(1.3) and u[3] == pytest.approx(1.7)
    # a ring with both |U| = 1 and sqrt 2 cells
    assert mo.ring_mean_u(nt, [1.0, 1.5])[0] == pytest.approx((1 + math.sqrt(2)) / 2, rel=1e-15)


def test_kpar_axis():
    k = mo.kpar_axis(8, rprime=2.0, dnu_c=0.5)
    assert k[4] == 0.0 and k[0] == pytest.approx(-4 * 2 * np.pi / (2.0 * 8 * 0.5))
    np.testing.assert_allclose(np.diff(k), 2 * np.pi / 8.0)


def test_cylindrical_binning_pins():
    """Constant planes give sum = value x count; the counts factor into the
    per-axis counts; the total over bins equals the sum over the covered
    delay pairs; a point-symmetric plane B(a, b) = B(-a, -b) gives a
    point-symmetric binned plane on symmetric edges."""
    nc = 12
    kpar = mo.kpar_axis(nc, 1.0, 1.0)
    edges = np.linspace(-2.0, 2.0, 5)  # k_par = a pi / 6: a = -3 .. 3 fall in [-2, 2)
    q = mo.axis_bins(kpar, edges)
    # a = -3, -2 -> [-2, -1); a = -1 -> [-1, 0); a = 0, 1 -> [0, 1); a = 2, 3 -> [1, 2)
    assert list(q) == [-1, -1, -1, 0, 0, 1, 2, 2, 3, 3, -1, -1]
    b3 = np.full((1, 2, nc, nc), 3.0)
    s, c = mo.bs_cylindrical(b3, kpar, edges)
    na = np.bincount(q[q >= 0], minlength=4)
    np.testing.assert_array_equal(c, np.outer(na, na))
    np.testing.assert_allclose(s, np.broadcast_to(3.0 * c, s.shape))
    r = np.random.default_rng(3)
    x = r.normal(size=(2, 3, nc, nc))
    s, c = mo.bs_cylindrical(x, kpar, edges)
    inside = q >= 0
    np.testing.assert_allclose(s.sum(axis=(-1, -2)), x[:, :, inside][:, :, :, inside].sum(axis=(-1, -2)))
    # point symmetry about a = b = 0 (index nc/2): reflect the indices 1 .. nc-1
    y = r.normal(size=(1, 1, nc, nc))
    ys = y.copy()
    ys[..., 1:, 1:] = 0.5 * (y[..., 1:, 1:] + y[..., 1:, 1:][..., ::-1, ::-1])
    e_sym = np.array([-1.6, -0.5, 0.5, 1.6])  # symmetric, kpar a = -1, 0, 1 and +-1.047
    s, c = mo.bs_cylindrical(ys, kpar, e_sym)
    np.testing.assert_allclose(s[0, 0], s[0, 0][::-1, ::-1], rtol=1e-13)


def _fp32_squared_decision(trips, kperp, kpar, k1_edges, n_mu, n_t, mistake=None):
    """A numpy FP32 emulation of a bin decision on squared quantities (the
    route a fast kernel takes): S_n in FP32, k1 by E_q = fl32(e_q^2) <= S1,
    t by S2 >= tau^2 S1, mu by N^2 >= 4 m^2 S1 S2 with N = S1 + S2 - S3.
    ``mistake`` plants an error to show the interval check catches it."""
    f = np.float32
    kp = np.asarray(kperp, np.float64).astype(f)
    kz = np.asarray(kpar, np.float64).astype(f)
    E = (np.asarray(k1_edges, np.float64) ** 2).astype(f)
    lo, hi = 0.5 - mo.SHAPE_TOL, 1.0 + mo.SHAPE_TOL
    tq = np.array([lo] + [0.5 + 0.5 * q / n_t for q in range(1, n_t)]) ** 2
    mq = 4 * np.array([lo] + [0.5 + 0.5 * q / n_mu for q in range(1, n_mu)] + [hi]) ** 2
    tq, mq = tq.astype(f), mq.astype(f)
    n_k1 = len(k1_edges) - 1
    cnt = np.zeros(n_k1 * n_mu * n_t, np.int64)
    ka, kb = kz[:, None], kz[None, :]
    kc = -(ka + kb)
    for (i, j, l) in trips:
        S = np.stack(np.broadcast_arrays(kp[i] * kp[i] + ka * ka, kp[j] * kp[j] + kb * kb,
                                         kp[l] * kp[l] + kc * kc))
        if mistake == "third_side_wrong_ring":
            S[2] = kp[j] * kp[j] + kc * kc
        S = np.sort(S, axis=0)[::-1]
        s1, s2, s3 = S
        N = (s1 + s2) - s3
        if mistake == "mu_sign":
            N = (s1 - s2) + s3
        P, N2 = s1 * s2, N * N
        ok = (s1 >= E[0]) & (s1 < E[-1]) & (s2 >= tq[0] * s1) & (N2 >= mq[0] * P) & (N2 <= mq[-1] * P)
        qk = np.searchsorted(E, s1, side="right") - 1
        qt = sum((s2 >= tq[q] * s1).astype(np.int64) for q in range(1, n_t))
        qm = sum((N2 >= mq[q] * P).astype(np.int64) for q in range(1, n_mu))
        q = np.where(ok, (qk * n_mu + qm) * n_t + qt, -1).ravel()
        cnt += np.bincount(q[q >= 0], minlength=cnt.size)
    return cnt.reshape(n_k1, n_mu, n_t)


def _interval_setup():
    r = np.random.default_rng(23)
    nb, nc = 6, 64
    kperp = np.sort(r.uniform(0.02, 0.4, nb))
    trips = [(i, j, l) for i in range(nb) for j in range(i, nb) for l in range(j, nb)][::3]
    kpar = mo.kpar_axis(nc, rprime=10.0, dnu_c=0.1)
    edges = np.geomspace(0.03, 3.0, 13)
    return trips, kperp, kpar, edges


def test_interval_holds_an_fp32_squared_decision():
    """The FP32 squared-length decision lands inside the interval of
    samples within 1e-5 of an edge, and the interval is narrow."""
    trips, kperp, kpar, edges = _interval_setup()
    iv = mo.monopole_interval(None, trips, kperp, kpar, edges, 5, 5, 2e-6, 1e-5,
                              model=(1.0, 1.0, -2.0))
    _, c = mo.bs_monopole(None, trips, kperp, kpar, edges, 5, 5, model=(1.0, 1.0, -2.0))
    assert np.all(iv["c_lo"] <= c) and np.all(c <= iv["c_hi"])
    c32 = _fp32_squared_decision(trips, kperp, kpar, edges, 5, 5)
    assert np.all(iv["c_lo"] <= c32) and np.all(c32 <= iv["c_hi"])
    assert iv["n_amb"] < 1e-3 * iv["n"]
    # samples on an edge in exact arithmetic are flagged: mu = 0.6 (the edge
    # of the first two mu bins) and k1 on a k1 edge
    q, amb, cand = mo.bin_candidates(np.array([1.0, edges[4]]), np.array([0.6, 0.75]),
                                     np.array([1.0, 0.75]), edges, 5, 5, 2e-6, 1e-5)
    assert amb.all() and q[0] >= 0 and q[1] >= 0
    assert len(set(cand[:, 0])) == 2 and len(set(cand[:, 1])) == 2


@pytest.mark.parametrize("mistake", ["mu_sign", "third_side_wrong_ring"])
def test_interval_rejects_planted_mistakes(mistake):
    trips, kperp, kpar, edges = _interval_setup()
    iv = mo.monopole_interval(None, trips, kperp, kpar, edges, 5, 5, 2e-6, 1e-5,
                              model=(1.0, 1.0, -2.0))
    c32 = _fp32_squared_decision(trips, kperp, kpar, edges, 5, 5, mistake=mistake)
    assert not (np.all(iv["c_lo"] <= c32) and np.all(c32 <= iv["c_hi"]))


# ---------------------------------------------------------------- multipoles

def test_legendre_against_library_and_parity():
    special = pytest.importorskip("scipy.special")
    x = np.linspace(-1.0, 1.0, 401)
    P = mo.legendre(6, x)
    for l in range(7):
        np.testing.assert_allclose(P[l], special.eval_legendre(l, x), rtol=0, atol=1e-14)
        assert P[l][-1] == pytest.approx(1.0, abs=1e-15)            # P_l(1) = 1
        np.testing.assert_allclose(P[l][::-1], (-1) ** l * P[l], atol=1e-15)
    # the orthogonality that makes (2l+1) <P_l B> the coefficient of P_l
    xg, wg = np.polynomial.legendre.leggauss(12)
    Pg = mo.legendre(4, xg)
    G = (Pg * wg) @ Pg.T
    np.testing.assert_allclose(G, np.diag(2.0 / (2 * np.arange(5) + 1)), atol=1e-14)


def test_mu1_against_explicit_vectors():
    """mu_1 = k_par / k of the largest side, from explicit 3D vectors whose
    sky-plane parts are random and whose third side closes the triangle."""
    r = np.random.default_rng(41)
    for _ in range(3000):
        pa, pb = r.normal(size=2), r.normal(size=2) * r.uniform(0.2, 2.0)
        za, zb = r.normal(size=2) * r.uniform(0.1, 5.0)
        vecs = [np.r_[pa, za], np.r_[pb, zb]]
        vecs.append(-(vecs[0] + vecs[1]))
        big = max(vecs, key=lambda v: np.dot(v, v))
        ref = big[2] / np.linalg.norm(big)
        S = [np.dot(v, v) for v in vecs]
        got = float(mo._mu1(S[0], S[1], S[2], za, zb))
        assert got == pytest.approx(ref, abs=1e-13)


def _brute_multipoles(b3d, trips, kperp, kpar, k1_edges, n_mu, n_t, lmax):
    """Per-sample loops: bins by linear search, the line-of-sight cosine of
    the longest side from its components, P_l from their closed forms."""
    closed = [lambda x: 1.0, lambda x: x, lambda x: (3 * x * x - 1) / 2,
              lambda x: (5 * x ** 3 - 3 * x) / 2, lambda x: (35 * x ** 4 - 30 * x * x + 3) / 8]
    n_k1 = len(k1_edges) - 1
    batch, _, nc, _ = b3d.shape
    sums = np.zeros((batch, lmax + 1, n_k1, n_mu, n_t))
    cnt = np.zeros((n_k1, n_mu, n_t), np.int64)
    tol = mo.SHAPE_TOL
    mu_e = [0.5 + 0.5 * q / n_mu for q in range(n_mu + 1)]
    t_e = [0.5 + 0.5 * q / n_t for q in range(n_t + 1)]
    lo = 1 if nc % 2 == 0 else 0  # the delay index -nc/2 has no reflection
    for p, (i, j, l) in enumerate(trips):
        for ia in range(lo, nc):
            for ib in range(lo, nc):
                z = [kpar[ia], kpar[ib], -(kpar[ia] + kpar[ib])]
                k = [math.sqrt(kperp[m] ** 2 + zz ** 2) for m, zz in zip((i, j, l), z)]
                order = sorted(range(3), key=lambda n: -k[n])  # stable: first of equal sides
                k1, k2, k3 = (k[n] for n in order)
                mu = (k1 * k1 + k2 * k2 - k3 * k3) / (2 * k1 * k2)
                t = k2 / k1
                if not (0.5 - tol <= mu <= 1 + tol and 0.5 - tol <= t <= 1 + tol):
                    continue
                mu, t = min(max(mu, 0.5), 1.0), min(max(t, 0.5), 1.0)
                qk = next((q for q in range(n_k1) if k1_edges[q] <= k1 < k1_edges[q + 1]), None)
                if qk is None:
                    continue
                qm = next(q for q in range(n_mu) if mu < mu_e[q + 1] or q == n_mu - 1)
                qt = next(q for q in range(n_t) if t < t_e[q + 1] or q == n_t - 1)
                x = z[order[0]] / k1
                cnt[qk, qm, qt] += 1
                for ll in range(lmax + 1):
                    sums[:, ll, qk, qm, qt] += (2 * ll + 1) * closed[ll](x) * b3d[:, p, ia, ib]
    return sums, cnt


@pytest.mark.parametrize("nc", [10, 9])
def test_multipoles_against_brute_force(nc):
    r = np.random.default_rng(12 + nc)
    nb = 4
    kperp = np.sort(r.uniform(0.05, 0.3, nb))
    trips = [(0, 0, 0), (0, 1, 1), (0, 1, 2), (1, 2, 3), (3, 3, 3)]
    kpar = mo.kpar_axis(nc, rprime=30.0, dnu_c=0.05)
    b3d = r.normal(size=(2, len(trips), nc, nc))
    edges = np.geomspace(0.04, 2.5, 7)
    s, c = mo.bs_multipoles(b3d, trips, kperp, kpar, edges, 5, 5, 4)
    s_b, c_b = _brute_multipoles(b3d, trips, kperp, kpar, edges, 5, 5, 4)
    np.testing.assert_array_equal(c, c_b)
    np.testing.assert_allclose(s, s_b, rtol=1e-11, atol=1e-11)
    assert c.sum() > 0 and np.abs(s[:, 1:]).max() > 0


def test_multipole_l0_is_the_monopole_for_odd_nc():
    """Odd nc: every delay index has its reflection, the multipole samples are
    the monopole's, and l = 0 is the monopole sum."""
    r = np.random.default_rng(3)
    nb, nc = 5, 15
    kperp = np.sort(r.uniform(0.05, 0.3, nb))
    trips = [(0, 1, 1), (1, 2, 3), (2, 3, 4), (4, 4, 4)]
    kpar = mo.kpar_axis(nc, rprime=20.0, dnu_c=0.05)
    b3d = r.normal(size=(1, len(trips), nc, nc))
    edges = np.geomspace(0.04, 2.5, 9)
    s, c = mo.bs_multipoles(b3d, trips, kperp, kpar, edges, 5, 5, 2)
    s0, c0 = mo.bs_monopole(b3d, trips, kperp, kpar, edges, 5, 5)
    np.testing.assert_array_equal(c, c0)
    np.testing.assert_allclose(s[:, 0], s0, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("nc", [16, 15])
def test_odd_multipoles_vanish_for_point_symmetric_b(nc):
    """B(-a, -b) = B(a, b) (the real part of a Hermitian 3D bispectrum): the
    reflection flips mu_1 and keeps the bin, so odd l cancel; even l do not."""
    r = np.random.default_rng(7)
    nb = 5
    kperp = np.sort(r.uniform(0.05, 0.3, nb))
    trips = [(0, 0, 1), (0, 2, 2), (1, 2, 3), (2, 4, 4)]
    kpar = mo.kpar_axis(nc, rprime=20.0, dnu_c=0.05)
    lo = nc % 2 == 0
    refl = np.r_[0, nc - np.arange(1, nc)] if lo else nc - 1 - np.arange(nc)
    np.testing.assert_array_equal(kpar[refl[lo:]], -kpar[lo:])
    b3d = r.normal(size=(1, len(trips), nc, nc))
    b3d = 0.5 * (b3d + b3d[:, :, refl][:, :, :, refl])
    edges = np.geomspace(0.04, 2.5, 9)
    s, c = mo.bs_multipoles(b3d, trips, kperp, kpar, edges, 5, 5, 4)
    scale = np.abs(b3d).max() * max(c.max(), 1) * 9
    assert np.abs(s[:, 1::2]).max() < 1e-13 * scale
    assert np.abs(s[:, 2]).max() > 1e-3 * np.abs(b3d).max()
    # the unpaired row of an even nc is left out: changing it changes nothing
    if lo:
        b3d[:, :, 0, :] += 1.0
        s_bad, _ = mo.bs_multipoles(b3d, trips, kperp, kpar, edges, 5, 5, 4)
        np.testing.assert_allclose(s_bad, s, atol=1e-12)


def test_multipole_interval_holds_the_fp64_decision():
    trips, kperp, kpar, edges = _interval_setup()
    r = np.random.default_rng(9)
    b3d = r.normal(size=(2, len(trips), kpar.size, kpar.size))
    iv = mo.multipole_interval(b3d, trips, kperp, kpar, edges, 5, 5, 3, 2e-6, 1e-5)
    s, c = mo.bs_multipoles(b3d, trips, kperp, kpar, edges, 5, 5, 3)
    assert np.all(iv["c_lo"] <= c) and np.all(c <= iv["c_hi"])
    assert np.all(np.abs(s - iv["s_sure"]) <= iv["s_amb"] + 1e-10)
    assert iv["n_amb"] < 1e-3 * iv["n"]
