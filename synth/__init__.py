"""Seeded synthetic inputs shared by the tests, the bench and the oracle.

This module holds no arithmetic of the estimator: it only draws inputs.  It
produces

* the validation sky of Section 4: a Gaussian random field ``g`` with power
  spectrum ``P(k) ~ k^slope`` on a periodic flat-sky box (two transverse axes
  of ``nt`` cells, one frequency axis of ``nc`` channels, unit cells), made
  non-Gaussian by the local transform of Eq. (mb1),
  ``delta = g + f_NG (g^2 - sigma^2)``;
* its gridded visibilities ``V(U_g, nu)``: the 2D discrete Fourier transform
  of each channel's sky plane (the flat-sky visibility of Section 3.1), stored
  centred, ``V[nu, v + nt/2, u + nt/2]``, complex, Hermitian
  (``V(-U) = V(U)^*``) because the sky is real;
* the channel flag pattern of Section 4 (periodic coarse-band flags) in the
  variant used by the flagged configuration: channel ``c`` flagged iff
  ``c mod 32`` is in ``{0, 1, 16, 30, 31}``;
* annular ring edges (linear and log spaced) in grid units of ``|U|``.

Random numbers come from numpy's Philox counter-based generator, seeded per
realisation, so the same seed gives the same sky on any machine.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "grf_power",
    "nongaussian_sky",
    "visibilities",
    "sky_visibilities",
    "flag_mask_coarse_band",
    "edges_linear",
    "edges_log",
    "rng",
]


def rng(seed: int) -> np.random.Generator:
    """Philox-backed generator for one realisation."""
    return np.random.Generator(np.random.Philox(int(seed)))


def _kmag(nt: int, nc: int) -> np.ndarray:
    """|k| on the periodic (nc, nt, nt) box, cells of unit size, axis order (z, y, x)."""
    kz = 2.0 * np.pi * np.fft.fftfreq(nc)
    ky = 2.0 * np.pi * np.fft.fftfreq(nt)
    kx = 2.0 * np.pi * np.fft.fftfreq(nt)
    return np.sqrt(kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2)


def grf_power(nt: int, nc: int, slope: float = -2.0, sigma: float = 0.5) -> np.ndarray:
    """Per-mode variance P(k) on the box, P(0) = 0, scaled so that the field
    variance (1/N) sum_k P(k) equals sigma^2.  Shape (nc, nt, nt)."""
    k = _kmag(nt, nc)
    p = np.zeros_like(k)
    nz = k > 0
    p[nz] = k[nz] ** slope
    p *= sigma**2 * k.size / p.sum()
    return p


def nongaussian_sky(nt: int, nc: int, seed: int, f_ng: float = 0.5, sigma: float = 0.5,
                    slope: float = -2.0) -> np.ndarray:
    """Real sky delta[nu, y, x] = g + f_NG (g^2 - sigma^2), Eq. (mb1).

    g = IDFT( sqrt(P) * DFT(w) ) with w white unit-variance noise, so that
    <g_hat(k) g_hat(k')> = N P(k) delta_{k+k'} and <g^2> = sigma^2.
    """
    w = rng(seed).standard_normal((nc, nt, nt))
    p = grf_power(nt, nc, slope, sigma)
    g = np.fft.ifftn(np.sqrt(p) * np.fft.fftn(w)).real
    return g + f_ng * (g * g - sigma**2)


def visibilities(sky: np.ndarray) -> np.ndarray:
    """V[nu, v + nt/2, u + nt/2] = sum_{x,y} sky[nu, y, x] exp(-2 pi i (u x + v y)/nt).

    Centred storage; cells with u or v = -nt/2 exist in the array but carry
    no Hermitian partner and are never binned by the estimator."""
    v = np.fft.fft2(sky, axes=(1, 2))
    return np.fft.fftshift(v, axes=(1, 2))


def sky_visibilities(nt: int, nc: int, seed: int, f_ng: float = 0.5, sigma: float = 0.5,
                     slope: float = -2.0, dtype=np.complex64) -> np.ndarray:
    """Visibilities of the validation sky, shape (nc, nt, nt)."""
    return visibilities(nongaussian_sky(nt, nc, seed, f_ng, sigma, slope)).astype(dtype)


def flag_mask_coarse_band(nc: int, flagged=(0, 1, 16, 30, 31), band: int = 32) -> np.ndarray:
    """uint8 [nc], 1 = channel flagged (periodic coarse-band pattern)."""
    c = np.arange(nc)
    return np.isin(c % band, np.asarray(flagged)).astype(np.uint8)


def edges_linear(nbins: int, u_max: float) -> np.ndarray:
    """nbins equal-width rings covering 0 <= |U| < u_max (U = 0 is never binned)."""
    return np.linspace(0.0, float(u_max), nbins + 1)


def edges_log(nbins: int, u_min: float, u_max: float) -> np.ndarray:
    """nbins log-spaced rings covering u_min <= |U| < u_max."""
    return np.geomspace(float(u_min), float(u_max), nbins + 1)


# ---------------------------------------------------------------------------
# Counter-based generator shared (by definition, not by code) with the GPU
# sky generator: Philox4x32 with 10 rounds (Salmon, Moraes, Dror & Shaw 2011,
# "Parallel random numbers: as easy as 1, 2, 3"), and Box-Muller normals.
# ---------------------------------------------------------------------------

_PH_M0, _PH_M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_PH_W0, _PH_W1 = np.uint64(0x9E3779B9), np.uint64(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32(counter, key, rounds: int = 10):
    """Philox4x32: counter uint64 array [..., 4] of 32-bit words, key [2].
    Each round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2,
    c = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); then k += (W0, W1)."""
    c = np.asarray(counter, dtype=np.uint64) & _MASK32
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0, k1 = np.uint64(int(key[0]) & 0xFFFFFFFF), np.uint64(int(key[1]) & 0xFFFFFFFF)
    for _ in range(rounds):
        p0 = _PH_M0 * c0
        p1 = _PH_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + _PH_W0) & _MASK32
        k1 = (k1 + _PH_W1) & _MASK32
    return np.stack([c0, c1, c2, c3], axis=-1)


def philox_normals(ncell: int, seed: int, realisation: int) -> np.ndarray:
    """Unit normals for cells 0..ncell-1: Philox call q (counter words
    q_lo, q_hi, r_lo, r_hi; key = seed lo, hi) gives four uint32 u; with
    u' = (u + 1/2) 2^-32, cells 4q, 4q+1 get Box-Muller of (u'0, u'1) and
    cells 4q+2, 4q+3 of (u'2, u'3):  sqrt(-2 ln a) (cos 2 pi b, sin 2 pi b)."""
    nq = (ncell + 3) // 4
    q = np.arange(nq, dtype=np.uint64)
    r = np.uint64(realisation)
    ctr = np.stack([q & _MASK32, q >> np.uint64(32), np.full(nq, r & _MASK32, np.uint64),
                    np.full(nq, r >> np.uint64(32), np.uint64)], axis=-1)
    out = philox4x32(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF))
    u = (out.astype(np.float64) + 0.5) * 2.0**-32
    rad0 = np.sqrt(-2.0 * np.log(u[:, 0]))
    rad1 = np.sqrt(-2.0 * np.log(u[:, 2]))
    n = np.empty((nq, 4))
    n[:, 0] = rad0 * np.cos(2 * np.pi * u[:, 1])
    n[:, 1] = rad0 * np.sin(2 * np.pi * u[:, 1])
    n[:, 2] = rad1 * np.cos(2 * np.pi * u[:, 3])
    n[:, 3] = rad1 * np.sin(2 * np.pi * u[:, 3])
    return n.reshape(-1)[:ncell]


def philox_sky_visibilities(nt: int, nc: int, seed: int, realisation: int, f_ng: float = 0.5,
                            sigma: float = 0.5, slope: float = -2.0) -> np.ndarray:
    """The validation sky of Eq. (mb1) drawn with the Philox normals above
    (same recipe as sky_visibilities, other random numbers): white noise
    w[z, y, x] = normals of cell (z nt + y) nt + x, g = IDFT(sqrt(P) DFT(w)),
    delta = g + f (g^2 - sigma^2), V[nu] = fftshift(DFT2(delta[nu])).
    complex128 (nc, nt, nt)."""
    w = philox_normals(nc * nt * nt, seed, realisation).reshape(nc, nt, nt)
    p = grf_power(nt, nc, slope, sigma)
    g = np.fft.ifftn(np.sqrt(p) * np.fft.fftn(w)).real
    d = g + f_ng * (g * g - sigma**2)
    return visibilities(d)
