"""Plain FP64 CPU oracle for the visibility-based MABS and 3D bispectrum
estimator of arXiv:2506.10526 (Section 3.2, Eqs. vg, iFT, iFT_I,
estimator_t, dft).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA library and never imports it; the product path never
imports this package.

Each function follows the paper's definition directly, with no FFT and no
reordering beyond what the definition states:

* ``ring_labels``      annular ring of each grid cell (Section 3.2, Section 4
                       ring layout); half-open rings, U = 0 never binned.
* ``weights``          W_g = 1/N_g for filled cells, 0 for empty ones, and 0 for
                       a flagged channel (Eq. vg and the text after Eq. iFT).
* ``mabs_full``        Eq. (estimator_t) for every ring triple i <= j <= l and
                       every ordered channel triple, evaluated as the sum over
                       closed grid triangles (C, FP64, ``enumerate.c``).
* ``collapse_fold``    ergodic collapse to (dnu1, dnu2) = (nu1-nu3, nu2-nu3) as
                       the mean over valid channel triples, with the lower
                       half-plane folded onto the upper one (Section 3.2 and
                       the discussion of Fig. Nv in Section 5).
* ``n_nu``             the sampling N_nu(dnu1, dnu2) of Fig. Nv.
* ``delay_dft``        Eq. (dft), the 2D DFT from (dnu1, dnu2) to (k_par1,
                       k_par2), written as the literal double sum.
* ``counts``           integer closed-triangle counts T(i, j, l).
* ``mabs_points`` / ``delta_points``  the same definitions at single sample
                       points, for grids too large for the full cube.
* ``analytic_mabs``    exact ensemble mean of the estimator for the Eq. (mb1)
                       test field on a periodic box (first-order term of
                       Eq. bsana plus the f_NG^3 loop term).
* ``gridding``         (module) nearest-grid-point gridding of raw
                       visibilities (Eq. vg) with the Hermitian mirror, and
                       the channel pre-averaging of Section 4.
* ``monopole``         (module) the 3D bispectrum monopole binned in triangle
                       size and shape: Eq. (shape), Eq. (bs_lm) at l = m = 0
                       and the (k1, mu, t) binning of Section 5, for
                       estimated values or for Eq. (bsana).

Pins (tests/test_oracle_pins.py) tie every function to something other than
itself: brute force, hand-worked cases, closed forms, invariants and the
analytic bispectrum.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from itertools import combinations_with_replacement

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile enumerate.c into oracle/_build/liboracle.so (gcc, OpenMP)."""
    src = os.path.join(_HERE, "enumerate.c")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src)):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                           "-o", tmp, src])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I = ctypes.c_int
            lib.orc_enumerate.argtypes = [I, I, I, P, P, P, P, I, P, P, P, P, P, I]
            lib.orc_counts.argtypes = [I, I, P, P, I]
            lib.orc_points.argtypes = [I, I, I, P, P, P, P, I, P, P, P, P, P, I]
            lib.orc_delta_points.argtypes = [I, I, I, P, P, P, P, I, I, I, P, P, P, P, I]
            lib.orc_delta_points_block.argtypes = [I, I, I, P, P, P, P, P, I, P, P, P, P, I]
            for f in (lib.orc_enumerate, lib.orc_counts, lib.orc_points, lib.orc_delta_points,
                      lib.orc_delta_points_block):
                f.restype = I
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# Section 3.2: rings and weights
# --------------------------------------------------------------------------

def ring_labels(nt: int, edges, occupancy=None) -> np.ndarray:
    """int32 [nt, nt] ring index of each centred cell, -1 if not binned.

    Cell (iv, iu) is the grid point U = (iu - nt/2, iv - nt/2).  Ring m holds
    the cells with e_m <= |U| < e_{m+1}, compared as |U|^2 (an exact integer)
    against e^2 in FP64.  U = 0 and cells with a component equal to -nt/2
    (no Hermitian partner on the grid) are never binned.  ``occupancy``
    (bool [nt, nt]) removes empty cells.
    """
    e = np.asarray(edges, dtype=np.float64)
    u = np.arange(nt) - nt // 2
    uu, vv = np.meshgrid(u, u, indexing="xy")  # uu[iv, iu] = u, vv[iv, iu] = v
    r2 = (uu.astype(np.int64) ** 2 + vv.astype(np.int64) ** 2).astype(np.float64)
    lab = np.full((nt, nt), -1, dtype=np.int32)
    e2 = e * e
    for m in range(len(e) - 1):
        sel = (r2 >= e2[m]) & (r2 < e2[m + 1])
        lab[sel] = m
    lab[(uu == 0) & (vv == 0)] = -1
    lab[(uu == -(nt // 2)) | (vv == -(nt // 2))] = -1
    if occupancy is not None:
        lab[~np.asarray(occupancy, dtype=bool)] = -1
    return lab


def weights(nc: int, nt: int, ngrid=None, chan_flags=None):
    """(W [nc, nt, nt], WN [nc, nt, nt]) in FP64.

    W = 1/N_g on filled cells and 0 on empty ones; a flagged channel has
    W = 0 everywhere, so its D and I fields vanish.  ``ngrid`` is None (every
    cell holds one visibility), [nt, nt] (same sampling in every channel) or
    [nc, nt, nt]."""
    if ngrid is None:
        n = np.ones((nc, nt, nt))
    else:
        n = np.broadcast_to(np.asarray(ngrid, dtype=np.float64), (nc, nt, nt)).copy()
    w = np.zeros_like(n)
    filled = n > 0
    w[filled] = 1.0 / n[filled]
    if chan_flags is not None:
        w[np.asarray(chan_flags, dtype=bool)] = 0.0
    return w, w * n


def ring_triples(nb: int):
    """Ring triples (i, j, l) with i <= j <= l, lexicographic."""
    return [t for t in combinations_with_replacement(range(nb), 3)]


# --------------------------------------------------------------------------
# Eq. (estimator_t)
# --------------------------------------------------------------------------

def mabs_full(vis, edges, ngrid=None, chan_flags=None, norm_A: float = 1.0,
              triples=None, nthreads: int = 0):
    """Binned MABS for every listed ring triple and every ordered channel triple.

    Returns a dict with
      ``B``   [ntrip, nc, nc, nc] complex: (1/A) num/den, NaN where den = 0
      ``num`` complex numerator sums, ``den`` real denominator sums,
      ``T``   [ntrip] closed-triangle counts (binned cells),
      ``triples`` the ring-triple list.
    Axis order of the cube: (nu1, nu2, nu3)."""
    vis = np.asarray(vis)
    nc, nt, _ = vis.shape
    e = np.asarray(edges, dtype=np.float64)
    nb = len(e) - 1
    lab = ring_labels(nt, e)
    w, wn = weights(nc, nt, ngrid, chan_flags)
    x = vis.astype(np.complex128) * w
    xre = np.ascontiguousarray(x.real.reshape(nc, -1))
    xim = np.ascontiguousarray(x.imag.reshape(nc, -1))
    y = np.ascontiguousarray(wn.reshape(nc, -1))
    trip = np.ascontiguousarray(np.array(triples if triples is not None else ring_triples(nb),
                                         dtype=np.int32).reshape(-1, 3))
    nt_ = trip.shape[0]
    num_re = np.empty((nt_, nc, nc, nc))
    num_im = np.empty_like(num_re)
    den = np.empty_like(num_re)
    tc = np.empty(nt_, dtype=np.int64)
    lab_c = np.ascontiguousarray(lab.reshape(-1))
    rc = _load().orc_enumerate(nt, nc, nb, _ptr(lab_c), _ptr(xre), _ptr(xim), _ptr(y), nt_,
                               _ptr(trip), _ptr(num_re), _ptr(num_im), _ptr(den), _ptr(tc),
                               int(nthreads))
    if rc != 0:
        raise MemoryError("orc_enumerate failed")
    num = num_re + 1j * num_im
    with np.errstate(invalid="ignore", divide="ignore"):
        B = np.where(den > 0, num / np.where(den > 0, den, 1.0), np.nan + 0j) / norm_A
    return {"B": B, "num": num, "den": den, "T": tc, "triples": [tuple(t) for t in trip]}


def counts(nt: int, edges, occupancy=None, nthreads: int = 0) -> np.ndarray:
    """T[i, j, l] (int64 [nb, nb, nb]): ordered closed triangles
    U_g1 + U_g2 + U_g3 = 0 with U_g1 in ring i, U_g2 in ring j, U_g3 in ring l."""
    e = np.asarray(edges, dtype=np.float64)
    nb = len(e) - 1
    lab = np.ascontiguousarray(ring_labels(nt, e, occupancy).reshape(-1))
    T = np.empty(nb * nb * nb, dtype=np.int64)
    if _load().orc_counts(nt, nb, _ptr(lab), _ptr(T), int(nthreads)) != 0:
        raise MemoryError("orc_counts failed")
    return T.reshape(nb, nb, nb)


def _prepare(vis, edges, ngrid, chan_flags):
    vis = np.asarray(vis)
    nc, nt, _ = vis.shape
    e = np.asarray(edges, dtype=np.float64)
    lab = np.ascontiguousarray(ring_labels(nt, e).reshape(-1))
    w, wn = weights(nc, nt, ngrid, chan_flags)
    x = vis.astype(np.complex128) * w
    return (nc, nt, len(e) - 1, lab, np.ascontiguousarray(x.real.reshape(nc, -1)),
            np.ascontiguousarray(x.imag.reshape(nc, -1)), np.ascontiguousarray(wn.reshape(nc, -1)))


def mabs_points(vis, edges, pts, ngrid=None, chan_flags=None, norm_A: float = 1.0,
                nthreads: int = 0):
    """Eq. (estimator_t) at single points (i, j, l, nu1, nu2, nu3).
    Returns (B complex [npts] with NaN where den = 0, T [npts])."""
    nc, nt, nb, lab, xre, xim, y = _prepare(vis, edges, ngrid, chan_flags)
    p = np.ascontiguousarray(np.asarray(pts, dtype=np.int32).reshape(-1, 6))
    n = p.shape[0]
    nr, ni, dn = np.empty(n), np.empty(n), np.empty(n)
    tc = np.empty(n, dtype=np.int64)
    _load().orc_points(nt, nc, nb, _ptr(lab), _ptr(xre), _ptr(xim), _ptr(y), n, _ptr(p),
                       _ptr(nr), _ptr(ni), _ptr(dn), _ptr(tc), int(nthreads))
    with np.errstate(invalid="ignore", divide="ignore"):
        B = np.where(dn > 0, (nr + 1j * ni) / np.where(dn > 0, dn, 1.0), np.nan) / norm_A
    return B, tc


def delta_points(vis, edges, pts, nu_lo: int = 0, nu_hi=None, ngrid=None, chan_flags=None,
                 norm_A: float = 1.0, nthreads: int = 0, block=None):
    """Folded collapsed MABS at points (i, j, l, d1, d2) for the channel window
    [nu_lo, nu_hi) of all three channels, or ``block`` = (nu1_lo, nu1_hi,
    nu2_lo, nu2_hi, nu3_lo, nu3_hi): the mean of Eq. (estimator_t) over the
    valid channel triples of the window with (nu1-nu3, nu2-nu3) = (d1, d2) or
    (-d1, -d2).  Returns (Bbar complex [npts], folded N_nu [npts])."""
    nc, nt, nb, lab, xre, xim, y = _prepare(vis, edges, ngrid, chan_flags)
    nu_hi = nc if nu_hi is None else int(nu_hi)
    blk = np.ascontiguousarray(np.asarray(
        block if block is not None else (nu_lo, nu_hi) * 3, dtype=np.int32))
    p = np.asarray(pts, dtype=np.int64).reshape(-1, 5)
    both = [p]
    neg = p.copy()
    neg[:, 3:] *= -1
    both.append(neg)
    q = np.ascontiguousarray(np.concatenate(both).astype(np.int32))
    n = q.shape[0]
    rr, ri = np.empty(n), np.empty(n)
    nv = np.empty(n, dtype=np.int64)
    rc = _load().orc_delta_points_block(nt, nc, nb, _ptr(lab), _ptr(xre), _ptr(xim), _ptr(y),
                                        _ptr(blk), n, _ptr(q), _ptr(rr), _ptr(ri), _ptr(nv),
                                        int(nthreads))
    if rc != 0:
        raise ValueError("orc_delta_points failed")
    m = p.shape[0]
    zero = (p[:, 3] == 0) & (p[:, 4] == 0)
    s = (rr[:m] + 1j * ri[:m]) + np.where(zero, 0.0, rr[m:] + 1j * ri[m:])
    c = nv[:m] + np.where(zero, 0, nv[m:])
    with np.errstate(invalid="ignore", divide="ignore"):
        out = np.where(c > 0, s / np.where(c > 0, c, 1), np.nan) / norm_A
    return out, c


# --------------------------------------------------------------------------
# Collapse to frequency separations, N_nu, Eq. (dft)
# --------------------------------------------------------------------------

def n_nu(valid) -> np.ndarray:
    """Unfolded N_nu[d1 + nc-1, d2 + nc-1]: number of channel triples
    (nu1, nu2, nu3), all valid, with nu1 - nu3 = d1 and nu2 - nu3 = d2."""
    v = np.asarray(valid, dtype=bool)
    nc = v.size
    out = np.zeros((2 * nc - 1, 2 * nc - 1), dtype=np.int64)
    for n3 in range(nc):
        if not v[n3]:
            continue
        for n1 in range(nc):
            if not v[n1]:
                continue
            for n2 in range(nc):
                if v[n2]:
                    out[n1 - n3 + nc - 1, n2 - n3 + nc - 1] += 1
    return out


def fold_plane(a: np.ndarray) -> np.ndarray:
    """Add the point reflection (d1, d2) -> (-d1, -d2) of a centred
    (2nc-1, 2nc-1) plane to itself, counting the origin once."""
    f = a + a[..., ::-1, ::-1]
    c = a.shape[-1] // 2
    f[..., c, c] = a[..., c, c]
    return f


def collapse_fold(B: np.ndarray):
    """Folded collapsed MABS from the full cube.

    B: [ntrip, nc, nc, nc] (nu1, nu2, nu3), NaN marking undefined triples.
    Returns (Bbar [ntrip, 2nc-1, 2nc-1] with NaN where no valid triple
    exists, folded count [ntrip, 2nc-1, 2nc-1]).  The plane is indexed
    [d1 + nc-1, d2 + nc-1] and is symmetric under (d1, d2) -> (-d1, -d2)."""
    B = np.asarray(B)
    ntrip, nc = B.shape[0], B.shape[1]
    s = np.zeros((ntrip, 2 * nc - 1, 2 * nc - 1), dtype=B.dtype)
    c = np.zeros((ntrip, 2 * nc - 1, 2 * nc - 1), dtype=np.int64)
    for n1 in range(nc):
        for n2 in range(nc):
            for n3 in range(nc):
                val = B[:, n1, n2, n3]
                ok = ~np.isnan(val)
                s[:, n1 - n3 + nc - 1, n2 - n3 + nc - 1] += np.where(ok, val, 0)
                c[:, n1 - n3 + nc - 1, n2 - n3 + nc - 1] += ok
    sf, cf = fold_plane(s), fold_plane(c)
    with np.errstate(invalid="ignore", divide="ignore"):
        bbar = np.where(cf > 0, sf / np.where(cf > 0, cf, 1), np.nan)
    return bbar, cf


def collapse_fold_ratio(num: np.ndarray, den: np.ndarray, norm_A: float = 1.0):
    """Folded collapse for per-channel sampling (reading: ratio of sums).

    With sampling that differs between channels the denominators of
    Eq. (estimator_t) differ between channel triples, and the collapse to
    (dnu1, dnu2) is read as the ratio of the summed numerators and the summed
    denominators over the channel triples at +-(d1, d2): with one sampling
    grid it equals the mean of the estimates (``collapse_fold``).
    num, den: [ntrip, nc, nc, nc] (nu1, nu2, nu3), as ``mabs_full`` returns
    them (zero where a channel is flagged or a cell empty).
    Returns the plane [ntrip, 2nc-1, 2nc-1], NaN where the summed
    denominator is zero."""
    ntrip, nc = num.shape[0], num.shape[1]
    n2 = 2 * nc - 1
    S = np.zeros((ntrip, n2, n2), dtype=num.dtype)
    D = np.zeros((ntrip, n2, n2))
    for n1 in range(nc):
        for n2_ in range(nc):
            for n3 in range(nc):
                S[:, n1 - n3 + nc - 1, n2_ - n3 + nc - 1] += num[:, n1, n2_, n3]
                D[:, n1 - n3 + nc - 1, n2_ - n3 + nc - 1] += den[:, n1, n2_, n3]
    Sf, Df = fold_plane(S), fold_plane(D)
    with np.errstate(invalid="ignore", divide="ignore"):
        return np.where(Df > 0, Sf / np.where(Df > 0, Df, 1.0), np.nan) / norm_A


def delay_dft(bbar: np.ndarray, nc: int, r: float = 1.0, rprime: float = 1.0,
              dnu_c: float = 1.0, variant: str = "half_open") -> np.ndarray:
    """Eq. (dft): B(a, b) = (r^2 r' dnu_c)^2 sum_{n,m} exp(-2 pi i (n a + m b)/nc)
    Bbar(n, m), a, b in [-nc/2, nc/2) (stored at index a + nc//2).

    The printed limits of the n, m sums, -nc/2 ... nc/2, give nc + 1 terms per
    axis with an nc-periodic kernel.  variant="half_open" (the reading used
    everywhere): n, m over the integers with -nc/2 <= n < nc/2, one full
    period (nc points).  variant="inclusive": both ends included (nc + 1
    points for even nc), reported beside it so the difference is visible.
    The 3D bispectrum is the real part: Bbar is point symmetric, so the
    imaginary part comes only from the unpaired edge row and column
    n, m = -nc/2 of the half-open range.  Separations where Bbar is undefined
    (no sampled triple) contribute nothing.  Input: centred (2nc-1, 2nc-1)
    planes [..., d1, d2].  Output: complex [..., nc, nc]."""
    bbar = np.asarray(bbar)
    h = nc // 2
    if variant == "half_open":
        n = np.arange(-h, nc - h)  # 2n >= -nc and 2n < nc
    elif variant == "inclusive":
        n = np.arange(-h, h + 1)
    else:
        raise ValueError(variant)
    sub = bbar[..., n + nc - 1, :][..., :, n + nc - 1]
    sub = np.where(np.isnan(sub), 0.0, sub)
    a = np.arange(-h, -h + nc)
    ker = np.exp(-2j * np.pi * np.outer(a, n) / nc)  # [a, n]
    out = ker @ sub @ ker.T  # sum over n then m: [..., a, b]
    return (r * r * rprime * dnu_c) ** 2 * out


# --------------------------------------------------------------------------
# Analytic ensemble mean for the Eq. (mb1) test field (periodic box)
# --------------------------------------------------------------------------

def loop_table(p: np.ndarray) -> np.ndarray:
    """L[k1, k3] = (1/N) sum_q P(q) P(k1 - q) P(k3 + q) for every pair of
    flattened wave-vector indices of the periodic box (N^2 entries; small
    boxes only).  For fixed k1 the q-sum is a cross-correlation of
    A(q) = P(q) P(k1 - q) with P, evaluated with the correlation theorem."""
    shp = p.shape
    N = p.size
    idx = np.indices(shp).reshape(3, -1).T
    ph = np.fft.fftn(p)
    out = np.empty((N, N))
    for t in range(N):
        k1 = idx[t]
        # A(q) = P(q) P(k1 - q): P(k1 - q) = P((k1 - q) mod shape)
        pm = p[(k1[0] - np.arange(shp[0]))[:, None, None] % shp[0],
               (k1[1] - np.arange(shp[1]))[None, :, None] % shp[1],
               (k1[2] - np.arange(shp[2]))[None, None, :] % shp[2]]
        a = p * pm
        corr = np.fft.ifftn(np.conj(np.fft.fftn(a)) * ph).real  # corr[k] = sum_q a(q) p(q + k)
        out[t] = corr.reshape(-1) / N
    return out


def box_bispectrum(p: np.ndarray, f_ng: float, k1, k2, ltab=None):
    """Exact discrete bispectrum of delta = g + f (g^2 - sigma^2) on a periodic
    box with per-mode variance p (shape (nz, ny, nx)), for integer wave-vector
    index arrays k1, k2 (..., 3) in (z, y, x) order, k3 = -k1 - k2:

      <d(k1) d(k2) d(k3)> / N = 2 f [P1 P2 + P2 P3 + P3 P1]            (Eq. bsana)
                                + 8 f^3 (1/N) sum_q P(q) P(k1 - q) P(k3 + q)

    The second line is the f^3 one-loop term that Eq. (bsana) drops (exact
    Wick sum: eight connected pairings, all equal after relabelling q); the
    f^2 term vanishes (odd moment of a Gaussian).  Valid for k1, k2, k3 != 0."""
    shp = np.array(p.shape)
    k1 = np.asarray(k1) % shp
    k2 = np.asarray(k2) % shp
    k3 = (-k1 - k2) % shp
    P1 = p[k1[..., 0], k1[..., 1], k1[..., 2]]
    P2 = p[k2[..., 0], k2[..., 1], k2[..., 2]]
    P3 = p[k3[..., 0], k3[..., 1], k3[..., 2]]
    tree = 2.0 * f_ng * (P1 * P2 + P2 * P3 + P3 * P1)
    if f_ng == 0.0:
        return tree
    if ltab is None:
        ltab = loop_table(p)
    f1 = (k1[..., 0] * shp[1] + k1[..., 1]) * shp[2] + k1[..., 2]
    f3 = (k3[..., 0] * shp[1] + k3[..., 1]) * shp[2] + k3[..., 2]
    return tree + 8.0 * f_ng**3 * ltab[f1, f3]


def analytic_mabs(nt: int, nc: int, edges, p: np.ndarray, f_ng: float, triples, d_pairs):
    """Exact ensemble mean of Eq. (estimator_t) (A = 1, every cell filled, no
    flags) for visibilities V[nu] = DFT2(delta[nu]) of the Eq. (mb1) field.

    For closed grid triangles (g1, g2, g3) and channels with separations
    (d1, d2) = (nu1 - nu3, nu2 - nu3):
      <V1 V2 V3> = (nt^2 / nc^2) sum_{kz1, kz2} B_box((g1,kz1), (g2,kz2), (g3,kz3))
                   exp(2 pi i (kz1 d1 + kz2 d2) / nc),  kz3 = -kz1 - kz2,
    which depends on the channels only through (d1, d2) (ergodicity, Section 2.2).
    The estimator is the plain mean of V1 V2 V3 over the ring triple's closed
    triangles.  Returns complex [len(triples), len(d_pairs)]."""
    lab = ring_labels(nt, edges)
    cells = {}
    for iv in range(nt):
        for iu in range(nt):
            m = lab[iv, iu]
            if m >= 0:
                cells.setdefault(m, []).append((iu - nt // 2, iv - nt // 2))
    ltab = loop_table(p) if f_ng != 0.0 else None
    kz = np.arange(nc)
    KZ1, KZ2 = np.meshgrid(kz, kz, indexing="ij")
    out = np.zeros((len(triples), len(d_pairs)), dtype=np.complex128)
    for ti, (i, j, l) in enumerate(triples):
        tris = []
        for (u1, v1) in cells.get(i, []):
            for (u2, v2) in cells.get(j, []):
                u3, v3 = -u1 - u2, -v1 - v2
                if abs(u3) < nt // 2 and abs(v3) < nt // 2 and lab[v3 + nt // 2, u3 + nt // 2] == l:
                    tris.append((u1, v1, u2, v2))
        if not tris:
            out[ti] = np.nan
            continue
        tr = np.array(tris)
        k1 = np.stack([np.broadcast_to(KZ1, KZ1.shape)[None].repeat(len(tr), 0),
                       np.broadcast_to(tr[:, 1, None, None], (len(tr), nc, nc)),
                       np.broadcast_to(tr[:, 0, None, None], (len(tr), nc, nc))], -1)
        k2 = np.stack([np.broadcast_to(KZ2, KZ2.shape)[None].repeat(len(tr), 0),
                       np.broadcast_to(tr[:, 3, None, None], (len(tr), nc, nc)),
                       np.broadcast_to(tr[:, 2, None, None], (len(tr), nc, nc))], -1)
        bb = box_bispectrum(p, f_ng, k1, k2, ltab)  # [ntri, kz1, kz2]
        mean_b = bb.mean(axis=0)
        for di, (d1, d2) in enumerate(d_pairs):
            ph = np.exp(2j * np.pi * (KZ1 * d1 + KZ2 * d2) / nc)
            out[ti, di] = (nt * nt / (nc * nc)) * np.sum(mean_b * ph)
    return out
