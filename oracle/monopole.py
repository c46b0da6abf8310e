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
* Binning arithmetic: the bin of a sample is decided in FP32, every
  operation rounded once (IEEE), in this order, which the GPU repeats so
  that bin indices agree bit for bit.  kperp and kpar are rounded to FP32;
  kpar_3 = -(kpar_1 + kpar_2); S_n = kperp_n^2 + kpar_n^2, sorted
  S1 >= S2 >= S3; K_n = sqrt(S_n); t = K2 / K1;
  mu = ((S1 + S2) - S3) / (2 (K1 K2)).  mu and t within 1e-6 of [0.5, 1]
  are clamped into it, samples further out (side lengths from ring means
  need not close) are dropped.  k1 bin q: e_q <= K1 < e_{q+1} (K1 widened
  to FP64, edges in FP64).  mu bin: floor((mu - 0.5) * (2 n_mu)) in FP32,
  the value 1 in the last bin; t alike.  Values and sums are FP64; the
  model of Eq. (bsana) takes the FP32 squared lengths widened to FP64.
"""
from __future__ import annotations

import numpy as np

SHAPE_TOL = 1e-6
F32 = np.float32


def triangle_shape(s1, s2, s3):
    """(k1, mu, t) of Eq. (shape) from the squared side lengths of a closed
    triangle (any order; arrays broadcast), computed in the inputs' floating
    type (FP64 for Python floats)."""
    arrs = np.broadcast_arrays(*(np.asarray(x) if isinstance(x, np.ndarray) and x.dtype == F32
                                 else np.asarray(x, np.float64) for x in (s1, s2, s3)))
    s = np.sort(np.stack(arrs), axis=0)[::-1]
    S1, S2, S3 = s[0], s[1], s[2]
    K1, K2 = np.sqrt(S1), np.sqrt(S2)
    t = K2 / K1
    two = S1.dtype.type(2.0)
    mu = ((S1 + S2) - S3) / (two * (K1 * K2))
    return K1, mu, t


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


def _bins(K1, mu, t, k1_edges, n_mu, n_t):
    """Flat bin index (k1, mu, t) of each FP32 sample, -1 where it falls outside."""
    e = np.asarray(k1_edges, np.float64)
    qk = np.searchsorted(e, K1.astype(np.float64), side="right") - 1
    ok = (qk >= 0) & (qk < e.size - 1)
    lo, hi = F32(0.5 - SHAPE_TOL), F32(1.0 + SHAPE_TOL)
    ok &= (mu >= lo) & (mu <= hi) & (t >= lo) & (t <= hi)
    half, one = F32(0.5), F32(1.0)
    muc = np.minimum(np.maximum(mu, half), one)
    tc = np.minimum(np.maximum(t, half), one)
    qm = np.minimum(np.floor((muc - half) * F32(2 * n_mu)).astype(np.int64), n_mu - 1)
    qt = np.minimum(np.floor((tc - half) * F32(2 * n_t)).astype(np.int64), n_t - 1)
    return np.where(ok, (qk * n_mu + qm) * n_t + qt, -1)


def bs_monopole(b3d, trips, kperp, kpar, k1_edges, n_mu: int, n_t: int, model=None):
    """Binned monopole sums and counts.

    b3d     [batch][n_planes][nc][nc] delay-space bispectrum, rows a + nc/2,
            columns b + nc/2 (or None with ``model``)
    trips   [n_planes] ring triples (i, j, l) of the planes
    kperp   [nbins] k_perp of each ring
    kpar    [nc] k_par of each row / column index
    model   None, or (f_ng, p_amp, p_index): bin Eq. (bsana) instead of b3d
    returns sums [batch][n_k1][n_mu][n_t], counts [n_k1][n_mu][n_t] (int64)
    """
    kpar = np.asarray(kpar, np.float64).astype(F32)
    kp = np.asarray(kperp, np.float64).astype(F32)
    nc = kpar.size
    n_k1 = len(k1_edges) - 1
    nbin = n_k1 * n_mu * n_t
    batch = 1 if b3d is None else b3d.shape[0]
    sums = np.zeros((batch, nbin))
    cnt = np.zeros(nbin, np.int64)
    ka = np.repeat(kpar[:, None], nc, axis=1)
    kb = np.repeat(kpar[None, :], nc, axis=0)
    kc = -(ka + kb)
    for p, (i, j, l) in enumerate(trips):
        S1 = kp[i] * kp[i] + ka * ka
        S2 = kp[j] * kp[j] + kb * kb
        S3 = kp[l] * kp[l] + kc * kc
        K1, mu, t = triangle_shape(S1, S2, S3)
        q = _bins(K1, mu, t, k1_edges, n_mu, n_t).ravel()
        sel = q >= 0
        cnt += np.bincount(q[sel], minlength=nbin)
        for b in range(batch):
            if model is None:
                v = np.asarray(b3d[b, p], np.float64).ravel()
            else:
                v = bsana(S1.astype(np.float64), S2.astype(np.float64), S3.astype(np.float64),
                          *model).ravel()
            sums[b] += np.bincount(q[sel], weights=v[sel], minlength=nbin)
    return sums.reshape(batch, n_k1, n_mu, n_t), cnt.reshape(n_k1, n_mu, n_t)


def _chunk(args):
    b3d, trips, kperp, kpar, k1_edges, n_mu, n_t, model = args
    return bs_monopole(b3d, trips, kperp, kpar, k1_edges, n_mu, n_t, model=model)


def bs_monopole_pool(trips, kperp, kpar, k1_edges, n_mu: int, n_t: int, model, workers: int = 16):
    """``bs_monopole`` of the model (no values) over many planes, the planes
    split across a spawn-started process pool: sums and counts of disjoint
    plane sets add."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    chunks = [trips[k::workers] for k in range(workers) if trips[k::workers]]
    args = [(None, c, kperp, kpar, k1_edges, n_mu, n_t, model) for c in chunks]
    with ProcessPoolExecutor(len(chunks), mp_context=mp.get_context("spawn")) as ex:
        parts = list(ex.map(_chunk, args))
    return sum(p[0] for p in parts), sum(p[1] for p in parts)


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
