"""Pins of the gridding oracle (oracle/gridding.py, Eq. vg): hand-placed
baselines, the Hermitian mirror, conservation of visibilities and counts,
flags, and pre-averaging as the sum of the unaveraged channels."""
import numpy as np

from oracle import gridding as gr


def test_hand_placed_baselines():
    nt = 8
    uv = np.array([[1.2, -0.4], [2.5, 1.49], [-0.5, 0.5], [3.7, 0.0], [-4.2, 1.0]])
    vis = np.array([[1 + 2j], [3 - 1j], [0.5j], [7.0], [9.0]])
    vg, ng = gr.grid_visibilities(uv, vis, None, nt)
    h = nt // 2
    # (1.2, -0.4) -> cell (1, 0); mirror (-1, 0)
    assert vg[0, 0 + h, 1 + h] == 1 + 2j and vg[0, 0 + h, -1 + h] == 1 - 2j
    # (2.5, 1.49) -> (3, 1) (halves round up); mirror (-3, -1)
    assert vg[0, 1 + h, 3 + h] == 3 - 1j and vg[0, -1 + h, -3 + h] == 3 + 1j
    # (-0.5, 0.5) -> (0, 1); mirror (0, -1)
    assert vg[0, 1 + h, 0 + h] == 0.5j and vg[0, -1 + h, 0 + h] == -0.5j
    # (3.7, 0) -> u = 4 = nt/2: outside; (-4.2, 1) -> u = -4: the unmirrored edge, dropped
    assert ng.sum() == 6
    assert gr.nearest_cell(np.array([-0.5, 0.5, -1.5, 2.4999]))[0] == 0
    assert list(gr.nearest_cell(np.array([-0.5, 0.5, -1.5, 2.4999]))) == [0, 1, -1, 2]


def test_hermitian_conservation_flags_and_averaging():
    r = np.random.default_rng(4)
    nt, nbl, nin = 16, 300, 12
    uv = r.uniform(-9.0, 9.0, size=(nbl, 2))
    vis = r.normal(size=(nbl, nin)) + 1j * r.normal(size=(nbl, nin))
    flags = (r.uniform(size=(nbl, nin)) < 0.2).astype(np.uint8)
    vg, ng = gr.grid_visibilities(uv, vis, flags, nt)
    h = nt // 2
    # Hermitian: V_g(-U) = V_g(U)*, N_g(-U) = N_g(U), on the mirrored part of the grid
    inner = (slice(None), slice(1, nt), slice(1, nt))
    np.testing.assert_allclose(vg[inner][:, ::-1, ::-1], np.conj(vg[inner]), atol=1e-12)
    np.testing.assert_array_equal(ng[inner][:, ::-1, ::-1], ng[inner])
    # conservation: each unflagged visibility inside the grid adds 2 counts and V + V*
    iu, iv = gr.nearest_cell(uv[:, 0]), gr.nearest_cell(uv[:, 1])
    inside = (np.abs(iu) < h) & (np.abs(iv) < h)
    use = inside[:, None] & (flags == 0)
    np.testing.assert_array_equal(ng.sum(axis=(1, 2)), 2 * use.sum(axis=0))
    np.testing.assert_allclose(vg.sum(axis=(1, 2)), 2 * np.where(use, vis.real, 0).sum(axis=0),
                               atol=1e-10)
    # pre-averaging by 4 equals the sum of the four unaveraged channels
    vg4, ng4 = gr.grid_visibilities(uv, vis, flags, nt, avg=4)
    np.testing.assert_allclose(vg4, vg.reshape(3, 4, nt, nt).sum(axis=1), atol=1e-12)
    np.testing.assert_array_equal(ng4, ng.reshape(3, 4, nt, nt).sum(axis=1))
    # every visibility flagged: an empty grid
    vg0, ng0 = gr.grid_visibilities(uv, vis, np.ones_like(flags), nt)
    assert not vg0.any() and not ng0.any()
