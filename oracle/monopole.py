"""Monopole of the 3D bispectrum binned in triangle size and shape.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it, and it never imports the CUDA library.

Definitions followed (arXiv:2506.10526):

* Section 2, Eq. (shape): for a closed triangle k1 + k2 + k3 = 0 with sides
  k1 >= k2 >= k3, the size is k1 and the shape is
      mu = -(k1 . k2) / (k1 k2),   t = k2 / k1,
  with 0.5 <= mu, t <= 1 and 2 mu t >= 1.  Because the vectors close,
  k1 . k2 = (k3^2 - k1^2 - k2^2) / 2, so mu = (k1^2 + k2^2 - k3^2) / (2 k1 k2)
  follows from the three squared lengths alone.
* Section 2: the 3D bispectrum B(k1perp, k2perp, k3perp, k1par, k2par) has
  k3par = -k1par - k2par; each side is k_n = sqrt(k_nperp^2 + k_npar^2).
* Section 2, Eq. (bs_lm) with l = m = 0: without redshift-space distortion
  the monopole is the orientation average of B at fixed (k1, mu, t); its
  discrete form (Section 5) is the mean of the estimated values whose
  triangles fall in a (k1, mu, t) bin: 12 logarithmic bins in k1 and 5
  linear bins in each of mu and t there.
* Section 3.2 / Eq. (dft): a delay index a in [-nc/2, nc/2) is
  k_par = 2 pi a / (r' nc dnu_c); the ring m of a triangle side gives
  k_perp = l / r = 2 pi U_m / r.
* Section 4, Eq. (bsana): B_ana = 2 f_NG [P(k1)P(k2) + P(k2)P(k3) + P(k3)P(k1)];
  binning it at the same discrete modes gives [B]_d of Section 5.

Readings (the paper leaves them open):

* Samples: every closable ring triple (T > 0) x every delay pair (a, b) of
  the Eq. (dft) output, a -> ring i (nu1), b -> ring j (nu2), the third
  component -a-b -> ring l.  The bin value is the unweighted mean.
* U_m of a ring is the mean |U| over its grid cells (grid units).
* Binning, as the definitions read, in FP64: k_n = sqrt(kperp_n^2 +
  kpar_n^2) with kpar_3 = -(kpar_1 + kpar_2); sides sorted k1 >= k2 >= k3;
  t = k2 / k1; mu = (k1^2 + k2^2 - k3^2) / (2 k1 k2).  The range
  0.5 <= mu, t <= 1 of Eq. (shape) holds for closed triangles; sides built
  from ring-mean k_perp close only approximately, and on the MWA-like grid
  (k_par >> k_perp) a large share of the samples are near-collinear with mu
  within 1e-4 above 1.  Samples within SHAPE_TOL = 1e-2 outside [0.5, 1] are
  therefore clamped into it and only those further out (sides that clearly
  cannot close) are dropped; few samples lie near that limit.  k1 bin
  q: e_q <= k1 < e_{q+1}; mu bin q: 0.5 + q / (2 n_mu) <= mu, the value 1
  in the last bin; t alike.  Values, sums and the model of Eq. (bsana) are
  FP64.
* Multipoles (Eq. bs_lm) with m = 0: the line of sight has p_z = mu_1 =
  k_par(side 1) / k1 in the triangle frame (Eq. orient), and the discrete
  form of Eq. (bs_lm) -- the integral over orientations taken as 4 pi times
  the mean over a bin's samples -- gives
  B_l^0 = sqrt(4 pi (2l+1)) <Y_l^0 B> = (2l+1) <P_l(mu_1) B>.  The azimuth
  that m != 0 needs depends on the triangle's handedness in the sky plane,
  which side lengths from ring means cannot fix (and is undefined for the
  collinear triangles).  Multipole samples leave out the delay row and
  column a, b = -nc/2 of an even nc, whose point reflections lie outside the
  grid, so the sample set is closed under (a, b) -> (-a, -b): mu_1 changes
  sign and the bin does not, and odd l vanish for a point-symmetric 3D
  bispectrum.
* ``bin_candidates`` lists, for each sample, every bin (or the drop, -1)
  reachable by moving k1 by a relative ``rel_k`` and mu, t by ``rel_s``
  about their FP64 values.  A kernel that decides bins in lower precision
  may disagree with ``bs_monopole`` only on samples with more than one
  candidate; the tests check GPU counts and sums against that interval.
"""
from __future__ import annotations

import numpy as np

SHAPE_TOL = 1e-2


def triangle_shape(s1, s2, s3):
    """(k1, mu, t) of Eq. (shape) in FP64 from the squared side lengths of a
    closed triangle (any order; arrays broadcast): sides k_n = sqrt(S_n)
    sorted k1 >= k2 >= k3, t = k2 / k1, mu = (k1^2 + k2^2 - k3^2) / (2 k1 k2)."""
    arrs = np.broadcast_arrays(*(np.asarray(x, np.float64) for x in (s1, s2, s3)))
    s = np.sort(np.stack(arrs), axis=0)[::-1]
    S1, S2, S3 = s[0], s[1], s[2]
    k1, k2 = np.sqrt(S1), np.sqrt(S2)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = k2 / k1
        mu = (S1 + S2 - S3) / (2.0 * k1 * k2)
    return k1, mu, t


def ring_mean_u(nt: int, edges, labels=None) -> np.ndarray:
    """U_m: mean |U| of the grid cells of each ring (grid units); the mid
    point of the ring's edges when it holds no cell."""
    from . import ring_labels
    lab = ring_labels(nt, edges) if labels is None else labels
    h = nt // 2
    v, u = np.meshgrid(np.arange(nt) - h, np.arange(nt) - h, indexing="ij")
    mag = np.sqrt(u.astype(np.float64) ** 2 + v.astype(np.float64) ** 2)
    e = np.asarray(edges, np.float64)
    out = np.empty(e.size - 1)
    for m in range(e.size - 1):
        sel = lab == m
        out[m] = mag[sel].mean() if sel.any() else 0.5 * (e[m] + e[m + 1])
    return out


def kpar_axis(nc: int, rprime: float = 1.0, dnu_c: float = 1.0) -> np.ndarray:
    """k_par of the Eq. (dft) output rows a + nc/2, a in [-nc/2, nc/2)."""
    a = np.arange(nc) - nc // 2
    return a * (2.0 * np.pi / (rprime * nc * dnu_c))


def bsana(S1, S2, S3, f_ng: float, p_amp: float, p_index: float):
    """Eq. (bsana) with P(k) = p_amp k^p_index, from squared side lengths."""
    P = [p_amp * np.power(np.asarray(S, np.float64), 0.5 * p_index) for S in (S1, S2, S3)]
    return 2.0 * f_ng * (P[0] * P[1] + P[1] * P[2] + P[2] * P[0])


def _bins(k1, mu, t, k1_edges, n_mu, n_t):
    """Flat bin index (k1, mu, t) of each sample (FP64), -1 where it is
    dropped or falls outside the k1 edges."""
    e = np.asarray(k1_edges, np.float64)
    qk = np.searchsorted(e, k1, side="right") - 1
    ok = (qk >= 0) & (qk < e.size - 1)
    lo, hi = 0.5 - SHAPE_TOL, 1.0 + SHAPE_TOL
    with np.errstate(invalid="ignore"):
        ok &= (mu >= lo) & (mu <= hi) & (t >= lo) & (t <= hi)
        muc = np.nan_to_num(np.clip(mu, 0.5, 1.0), nan=0.5)
        tc = np.nan_to_num(np.clip(t, 0.5, 1.0), nan=0.5)
    qm = np.minimum(np.floor((muc - 0.5) * (2 * n_mu)).astype(np.int64), n_mu - 1)
    qt = np.minimum(np.floor((tc - 0.5) * (2 * n_t)).astype(np.int64), n_t - 1)
    return np.where(ok, (qk * n_mu + qm) * n_t + qt, -1)


def _plane_squares(kp, kpar, i, j, l):
    """Squared sides S1, S2, S3 [nc][nc] of ring triple (i, j, l) at every
    delay pair (a, b): kpar_1 = kpar[a], kpar_2 = kpar[b], kpar_3 = -(sum)."""
    ka = kpar[:, None]
    kb = kpar[None, :]
    kc = -(ka + kb)
    S1 = np.broadcast_to(kp[i] ** 2 + ka ** 2, kc.shape)
    S2 = np.broadcast_to(kp[j] ** 2 + kb ** 2, kc.shape)
    S3 = kp[l] ** 2 + kc ** 2
    return S1, S2, S3


def bs_monopole(b3d, trips, kperp, kpar, k1_edges, n_mu: int, n_t: int, model=None):
    """Binned monopole sums and counts (FP64 throughout).

    b3d     [batch][n_planes][nc][nc] delay-space bispectrum, rows a + nc/2,
            columns b + nc/2 (or None with ``model``)
    trips   [n_planes] ring triples (i, j, l) of the planes
    kperp   [nbins] k_perp of each ring
    kpar    [nc] k_par of each row / column index
    model   None, or (f_ng, p_amp, p_index): bin Eq. (bsana) instead of b3d
    returns sums [batch][n_k1][n_mu][n_t], counts [n_k1][n_mu][n_t] (int64)
    """
    kpar = np.asarray(kpar, np.float64)
    kp = np.asarray(kperp, np.float64)
    n_k1 = len(k1_edges) - 1
    nbin = n_k1 * n_mu * n_t
    batch = 1 if b3d is None else b3d.shape[0]
    sums = np.zeros((batch, nbin))
    cnt = np.zeros(nbin, np.int64)
    for p, (i, j, l) in enumerate(trips):
        S1, S2, S3 = _plane_squares(kp, kpar, i, j, l)
        k1, mu, t = triangle_shape(S1, S2, S3)
        q = _bins(k1, mu, t, k1_edges, n_mu, n_t).ravel()
        sel = q >= 0
        cnt += np.bincount(q[sel], minlength=nbin)
        for b in range(batch):
            if model is None:
                v = np.asarray(b3d[b, p], np.float64).ravel()
            else:
                v = bsana(S1, S2, S3, *model).ravel()
            sums[b] += np.bincount(q[sel], weights=v[sel], minlength=nbin)
    return sums.reshape(batch, n_k1, n_mu, n_t), cnt.reshape(n_k1, n_mu, n_t)


def legendre(lmax: int, x):
    """P_0(x) .. P_lmax(x) by Bonnet's recursion (l+1) P_{l+1} = (2l+1) x P_l - l P_{l-1}."""
    x = np.asarray(x, np.float64)
    P = [np.ones_like(x), x.copy()]
    for l in range(1, lmax):
        P.append(((2 * l + 1) * x * P[l] - l * P[l - 1]) / (l + 1))
    return np.stack(P[:lmax + 1])


def _mu1(S1, S2, S3, kpar_a, kpar_b):
    """mu_1 = k_par / k of the largest side (ties: the first of the sides
    in the order 1, 2, 3, as a stable sort gives)."""
    kc = -(kpar_a + kpar_b)
    S = np.stack(np.broadcast_arrays(S1, S2, S3))
    Z = np.stack(np.broadcast_arrays(kpar_a, kpar_b, kc))
    k = np.argmax(S, axis=0)  # first maximum
    s1 = np.take_along_axis(S, k[None], axis=0)[0]
    z1 = np.take_along_axis(Z, k[None], axis=0)[0]
    return z1 / np.sqrt(s1)


def paired_mask(nc: int) -> np.ndarray:
    """Delay indices whose point reflection is on the grid (all but a = -nc/2
    of an even nc)."""
    m = np.ones(nc, bool)
    if nc % 2 == 0:
        m[0] = False
    return m


def bs_multipoles(b3d, trips, kperp, kpar, k1_edges, n_mu: int, n_t: int, lmax: int):
    """Binned m = 0 multipoles: sums [batch][lmax+1][n_k1][n_mu][n_t] of
    (2l+1) P_l(mu_1) B over the paired samples of each bin, and their counts
    [n_k1][n_mu][n_t]; B_l^0 = sums / counts (FP64 throughout)."""
    kpar = np.asarray(kpar, np.float64)
    kp = np.asarray(kperp, np.float64)
    nc = kpar.size
    n_k1 = len(k1_edges) - 1
    nbin = n_k1 * n_mu * n_t
    batch = b3d.shape[0]
    sums = np.zeros((batch, lmax + 1, nbin))
    cnt = np.zeros(nbin, np.int64)
    pm = paired_mask(nc)
    keep = (pm[:, None] & pm[None, :]).ravel()
    ka = np.broadcast_to(kpar[:, None], (nc, nc))
    kb = np.broadcast_to(kpar[None, :], (nc, nc))
    wl = (2 * np.arange(lmax + 1) + 1)[:, None]
    for p, (i, j, l) in enumerate(trips):
        S1, S2, S3 = _plane_squares(kp, kpar, i, j, l)
        k1, mu, t = triangle_shape(S1, S2, S3)
        q = _bins(k1, mu, t, k1_edges, n_mu, n_t).ravel()
        sel = (q >= 0) & keep
        W = wl * legendre(lmax, _mu1(S1, S2, S3, ka, kb).ravel())  # [lmax+1][nc*nc]
        cnt += np.bincount(q[sel], minlength=nbin)
        for b in range(batch):
            v = np.asarray(b3d[b, p], np.float64).ravel()
            for ll in range(lmax + 1):
                sums[b, ll] += np.bincount(q[sel], weights=(W[ll] * v)[sel], minlength=nbin)
    return sums.reshape(batch, lmax + 1, n_k1, n_mu, n_t), cnt.reshape(n_k1, n_mu, n_t)


def multipole_interval(b3d, trips, kperp, kpar, k1_edges, n_mu: int, n_t: int, lmax: int,
                       rel_k: float, rel_s: float):
    """As ``monopole_interval`` for the multipole sums: per bin the counts of
    the sure and reachable samples, the sums over the sure samples, and the
    sums of |(2l+1) P_l(mu_1) B| over the ambiguous samples that can reach
    the bin (paired samples only)."""
    kpar = np.asarray(kpar, np.float64)
    kp = np.asarray(kperp, np.float64)
    nc = kpar.size
    n_k1 = len(k1_edges) - 1
    nbin = n_k1 * n_mu * n_t
    batch = b3d.shape[0]
    c_lo = np.zeros(nbin, np.int64)
    c_hi = np.zeros(nbin, np.int64)
    s_sure = np.zeros((batch, lmax + 1, nbin))
    s_amb = np.zeros((batch, lmax + 1, nbin))
    pm = paired_mask(nc)
    keep = (pm[:, None] & pm[None, :]).ravel()
    ka = np.broadcast_to(kpar[:, None], (nc, nc))
    kb = np.broadcast_to(kpar[None, :], (nc, nc))
    wl = (2 * np.arange(lmax + 1) + 1)[:, None]
    n_amb = 0
    n_all = 0
    for p, (i, j, l) in enumerate(trips):
        S1, S2, S3 = _plane_squares(kp, kpar, i, j, l)
        k1, mu, t = triangle_shape(S1, S2, S3)
        q, amb, cand = bin_candidates(k1, mu, t, k1_edges, n_mu, n_t, rel_k, rel_s)
        n_all += int(keep.sum())
        W = wl * legendre(lmax, _mu1(S1, S2, S3, ka, kb).ravel())
        amb_k = amb & keep
        n_amb += int(amb_k.sum())
        sure = (q >= 0) & ~amb & keep
        c_lo += np.bincount(q[sure], minlength=nbin)
        ai = np.flatnonzero(amb)            # columns of cand
        kc = keep[ai]
        idx = np.broadcast_to(np.arange(cand.shape[1])[None, :], cand.shape)
        ok = (cand >= 0) & kc[None, :]
        pairs = np.unique(np.stack([idx[ok], cand[ok]]), axis=1)
        c_hi += np.bincount(pairs[1], minlength=nbin)
        for b in range(batch):
            v = np.asarray(b3d[b, p], np.float64).ravel()
            for ll in range(lmax + 1):
                wv = W[ll] * v
                s_sure[b, ll] += np.bincount(q[sure], weights=wv[sure], minlength=nbin)
                s_amb[b, ll] += np.bincount(pairs[1], weights=np.abs(wv[ai])[pairs[0]],
                                            minlength=nbin)
    c_hi += c_lo
    shape = (n_k1, n_mu, n_t)
    return {"c_lo": c_lo.reshape(shape), "c_hi": c_hi.reshape(shape),
            "s_sure": s_sure.reshape((batch, lmax + 1) + shape),
            "s_amb": s_amb.reshape((batch, lmax + 1) + shape), "n_amb": n_amb, "n": n_all}


def bin_candidates(k1, mu, t, k1_edges, n_mu: int, n_t: int, rel_k: float, rel_s: float):
    """Bins a sample can take when k1 moves by a relative ``rel_k`` and mu, t
    by ``rel_s`` (absolute; both lie near [0.5, 1]) about their FP64 values
    (t never above 1: the sides are sorted).

    Returns (q, amb, cand): q the FP64 bin (-1 dropped), amb a mask of the
    samples with more than one candidate, cand [27][n_amb] the candidate bins
    of those samples (with repeats; -1 = dropped)."""
    k1, mu, t = (np.asarray(x, np.float64).ravel() for x in (k1, mu, t))
    q = _bins(k1, mu, t, k1_edges, n_mu, n_t)
    amb = np.zeros(q.shape, bool)

    def tmove(tt, dt):  # t = k2 / k1 <= 1 holds for sorted sides in any precision
        return np.minimum(tt + dt, 1.0) if dt > 0 else tt + dt

    for fk in (1 - rel_k, 1 + rel_k):
        amb |= _bins(k1 * fk, mu, t, k1_edges, n_mu, n_t) != q
    for dm in (-rel_s, rel_s):
        amb |= _bins(k1, mu + dm, t, k1_edges, n_mu, n_t) != q
        amb |= _bins(k1, mu, tmove(t, dm), k1_edges, n_mu, n_t) != q
    ka, ma, ta = k1[amb], mu[amb], t[amb]
    cand = np.stack([_bins(ka * fk, ma + dm, tmove(ta, dt), k1_edges, n_mu, n_t)
                     for fk in (1 - rel_k, 1.0, 1 + rel_k) for dm in (-rel_s, 0.0, rel_s)
                     for dt in (-rel_s, 0.0, rel_s)])
    return q, amb, cand


def monopole_interval(b3d, trips, kperp, kpar, k1_edges, n_mu: int, n_t: int, rel_k: float,
                      rel_s: float, model=None):
    """What a kernel whose bin decision may differ from the FP64 one within
    ``rel_k`` and ``rel_s`` (see ``bin_candidates``) can return.

    returns dict with, per bin, ``c_lo`` (samples whose only candidate is the
    bin), ``c_hi`` (samples having the bin among their candidates), ``s_sure``
    [batch][bin] (sums over the first set), ``s_amb`` [batch][bin] (sums of
    |value| over ambiguous samples that can reach the bin), and the numbers
    of samples ``n_amb`` and ``n`` (all samples)."""
    kpar = np.asarray(kpar, np.float64)
    kp = np.asarray(kperp, np.float64)
    n_k1 = len(k1_edges) - 1
    nbin = n_k1 * n_mu * n_t
    batch = 1 if b3d is None else b3d.shape[0]
    c_lo = np.zeros(nbin, np.int64)
    c_hi = np.zeros(nbin, np.int64)
    s_sure = np.zeros((batch, nbin))
    s_amb = np.zeros((batch, nbin))
    n_amb = 0
    n_all = 0
    for p, (i, j, l) in enumerate(trips):
        S1, S2, S3 = _plane_squares(kp, kpar, i, j, l)
        k1, mu, t = triangle_shape(S1, S2, S3)
        q, amb, cand = bin_candidates(k1, mu, t, k1_edges, n_mu, n_t, rel_k, rel_s)
        n_all += q.size
        n_amb += int(amb.sum())
        sure = (q >= 0) & ~amb
        c_lo += np.bincount(q[sure], minlength=nbin)
        # distinct candidate bins per ambiguous sample
        idx = np.broadcast_to(np.arange(cand.shape[1])[None, :], cand.shape).ravel()
        cb = cand.ravel()
        keep = cb >= 0
        pairs = np.unique(np.stack([idx[keep], cb[keep]]), axis=1)
        c_hi += np.bincount(pairs[1], minlength=nbin)
        for b in range(batch):
            if model is None:
                v = np.asarray(b3d[b, p], np.float64).ravel()
            else:
                v = bsana(S1, S2, S3, *model).ravel()
            s_sure[b] += np.bincount(q[sure], weights=v[sure], minlength=nbin)
            s_amb[b] += np.bincount(pairs[1], weights=np.abs(v[amb])[pairs[0]], minlength=nbin)
    c_hi += c_lo
    shape = (n_k1, n_mu, n_t)
    return {"c_lo": c_lo.reshape(shape), "c_hi": c_hi.reshape(shape),
            "s_sure": s_sure.reshape((batch,) + shape), "s_amb": s_amb.reshape((batch,) + shape),
            "n_amb": n_amb, "n": n_all}


def _chunk(args):
    fn, b3d, trips, kperp, kpar, k1_edges, n_mu, n_t, model, rel = args
    if fn == "interval":
        return monopole_interval(b3d, trips, kperp, kpar, k1_edges, n_mu, n_t, *rel, model=model)
    return bs_monopole(b3d, trips, kperp, kpar, k1_edges, n_mu, n_t, model=model)


def _pool(fn, trips, kperp, kpar, k1_edges, n_mu, n_t, model, rel, workers):
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    chunks = [trips[k::workers] for k in range(workers) if trips[k::workers]]
    args = [(fn, None, c, kperp, kpar, k1_edges, n_mu, n_t, model, rel) for c in chunks]
    with ProcessPoolExecutor(len(chunks), mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_chunk, args))


def bs_monopole_pool(trips, kperp, kpar, k1_edges, n_mu: int, n_t: int, model, workers: int = 16):
    """``bs_monopole`` of the model (no values) over many planes, the planes
    split across a spawn-started process pool: sums and counts of disjoint
    plane sets add."""
    parts = _pool("plain", trips, kperp, kpar, k1_edges, n_mu, n_t, model, None, workers)
    return sum(p[0] for p in parts), sum(p[1] for p in parts)


def monopole_interval_pool(trips, kperp, kpar, k1_edges, n_mu: int, n_t: int, model,
                           rel_k: float, rel_s: float, workers: int = 16):
    """``monopole_interval`` of the model over many planes in a spawn-started
    process pool (every field adds over disjoint plane sets)."""
    parts = _pool("interval", trips, kperp, kpar, k1_edges, n_mu, n_t, model, (rel_k, rel_s),
                  workers)
    return {k: sum(p[k] for p in parts) for k in parts[0]}


def axis_bins(kpar, edges) -> np.ndarray:
    """Bin of each delay index along one k_par axis: q with e_q <= k_par < e_{q+1},
    -1 outside (FP64 comparisons)."""
    e = np.asarray(edges, np.float64)
    q = np.searchsorted(e, np.asarray(kpar, np.float64), side="right") - 1
    return np.where((q >= 0) & (q < e.size - 1), q, -1)


def bs_cylindrical(b3d, kpar, edges):
    """The 3D bispectrum of each plane binned on a grid in the (k_par1,
    k_par2) plane (Section 5, the binning behind Fig. cylbs): sums
    [batch][n_planes][n][n] over the delay pairs (a, b) whose k_par(a),
    k_par(b) fall in bins (q, r), and counts [n][n] of those pairs (the same
    for every plane).  The bin value is sum / count."""
    q = axis_bins(kpar, edges)
    n = len(edges) - 1
    batch, npl, nc, _ = b3d.shape
    sums = np.zeros((batch, npl, n, n))
    cnt = np.zeros((n, n), np.int64)
    for a in range(nc):
        if q[a] < 0:
            continue
        for b in range(nc):
            if q[b] < 0:
                continue
            cnt[q[a], q[b]] += 1
            sums[:, :, q[a], q[b]] += b3d[:, :, a, b]
    return sums, cnt
