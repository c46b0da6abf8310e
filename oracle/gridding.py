"""Gridding of raw visibilities onto the uv grid (Eq. vg) and channel
pre-averaging (Section 4).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import it, and it never imports the CUDA library.

Definitions followed (arXiv:2506.10526):

* Section 3.2, Eq. (vg): on a square grid of spacing Delta U_g, every
  visibility V(U_i, nu) goes to the grid point U_g nearest to U_i:
  V_g(nu) = sum_i w(U_g - U_i) V(U_i, nu) F(U_i, nu), with w = 1 for the
  nearest grid point and 0 otherwise, F = 0 for flagged data and 1 otherwise,
  and N_g(nu) = sum_i w(U_g - U_i) F(U_i, nu) the number of visibilities
  that reach U_g.
* Section 4: four consecutive channels are collapsed into one (768 -> 192
  channels at 160 kHz).

Readings (the paper leaves them open):

* Baseline coordinates are in grid units (U / Delta U_g).  The nearest grid
  point of u is floor(u + 1/2) in FP64, and likewise for v.
* The sky is real, so V(-U) = V(U)*: each unflagged visibility also adds its
  conjugate at the mirrored cell -g (the mirror of the nearest cell, which
  keeps the grid Hermitian even for a baseline at a half-integer).
  Visibilities whose cell has |u| or |v| >= N_t / 2 (outside the centred
  grid, or at the -N_t/2 edge that has no mirror) are dropped.
* Channel pre-averaging by a factor ``avg``: input channel c feeds output
  channel c // avg, V_g and N_g summed over the avg inputs.  The estimator
  then weights V_g by 1 / N_g, which gives the mean over all contributing
  visibilities of the avg channels.
* Output layout: V_g complex [nchan][N_t][N_t] and N_g [nchan][N_t][N_t],
  centred (index u + N_t/2, v + N_t/2; row index v), the layout bs_grid_load
  reads.
"""
from __future__ import annotations

import numpy as np


def nearest_cell(u: np.ndarray) -> np.ndarray:
    """Nearest grid point of FP64 coordinates in grid units."""
    return np.floor(np.asarray(u, np.float64) + 0.5).astype(np.int64)


def grid_visibilities(uv, vis, flags, nt: int, avg: int = 1):
    """Eq. (vg) with the Hermitian mirror and channel pre-averaging.

    uv     [nbl][2] FP64 baseline (u, v) in grid units
    vis    [nbl][nchan_in] complex visibilities
    flags  [nbl][nchan_in] (1 = flagged) or None
    returns (V_g complex128 [nchan][nt][nt], N_g float64 [nchan][nt][nt]),
    nchan = nchan_in // avg
    """
    uv = np.asarray(uv, np.float64)
    vis = np.asarray(vis)
    nbl, nin = vis.shape
    nch = nin // avg
    h = nt // 2
    iu, iv = nearest_cell(uv[:, 0]), nearest_cell(uv[:, 1])
    inside = (np.abs(iu) < h) & (np.abs(iv) < h)
    vg = np.zeros((nch, nt, nt), np.complex128)
    ng = np.zeros((nch, nt, nt))
    for c in range(nch * avg):
        ok = inside.copy()
        if flags is not None:
            ok &= np.asarray(flags)[:, c] == 0
        o = c // avg
        for sgn, val in ((1, vis[ok, c]), (-1, np.conj(vis[ok, c]))):
            np.add.at(vg[o], (sgn * iv[ok] + h, sgn * iu[ok] + h), val)
            np.add.at(ng[o], (sgn * iv[ok] + h, sgn * iu[ok] + h), 1.0)
    return vg, ng
