"""Pins of the counter-based input generator (synth.philox4x32,
synth.philox_normals, synth.philox_sky_visibilities) that the GPU sky
generator is compared with: the published Philox4x32-10 known-answer
vectors, the distribution of the Box-Muller normals, and the recipe of the
sky against the numpy-seeded one on the same noise."""
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    rows = _kat()
    assert len(rows) == 3
    for ctr, key, want in rows:
        got = synth.philox4x32(np.array([ctr], dtype=np.uint64), key)[0]
        assert [int(x) for x in got] == want


def test_philox_counter_words_are_distinct_inputs():
    """Changing any one counter word or key word changes every output word."""
    base = synth.philox4x32(np.array([[1, 2, 3, 4]], dtype=np.uint64), (5, 6))[0]
    for pos in range(4):
        c = [1, 2, 3, 4]
        c[pos] ^= 1
        o = synth.philox4x32(np.array([c], dtype=np.uint64), (5, 6))[0]
        assert np.all(o != base)
    o = synth.philox4x32(np.array([[1, 2, 3, 4]], dtype=np.uint64), (5, 7))[0]
    assert np.all(o != base)


def test_box_muller_normals_are_standard_normal():
    n = synth.philox_normals(1 << 20, 2024, 3)
    assert abs(n.mean()) < 5e-3
    assert abs(n.var() - 1) < 5e-3
    assert abs(np.mean(n**4) - 3) < 0.03  # Gaussian kurtosis
    # fraction beyond 2 sigma: 2 (1 - Phi(2)) = 0.0455
    assert abs(np.mean(np.abs(n) > 2) - 0.0455) < 1.5e-3
    # the pair (cos, sin) of one call is uncorrelated
    assert abs(np.mean(n[0::4] * n[1::4])) < 1e-2


def test_normals_follow_cell_and_realisation_counters():
    """cells 4q..4q+3 come from call q; realisation r is counter words 2, 3."""
    a = synth.philox_normals(64, 9, 0)
    b = synth.philox_normals(128, 9, 0)
    np.testing.assert_array_equal(a, b[:64])
    c = synth.philox_normals(64, 9, 1)
    assert not np.any(a == c)
    o = synth.philox4x32(np.array([[5, 0, 1, 0]], dtype=np.uint64), (9, 0))[0]
    u = (o.astype(np.float64) + 0.5) * 2.0**-32
    want = np.sqrt(-2 * np.log(u[2])) * np.sin(2 * np.pi * u[3])
    assert c[4 * 5 + 3] == want


def test_philox_sky_is_hermitian_and_follows_the_recipe():
    nt, nc, seed, r = 16, 6, 4, 2
    v = synth.philox_sky_visibilities(nt, nc, seed, r)
    h = nt // 2
    inner = v[:, 1:, 1:]
    np.testing.assert_allclose(inner, np.conj(inner[:, ::-1, ::-1]), atol=1e-12)
    # same recipe as the numpy-seeded sky: redo it on the same white noise
    w = synth.philox_normals(nc * nt * nt, seed, r).reshape(nc, nt, nt)
    p = synth.grf_power(nt, nc)
    g = np.fft.ifftn(np.sqrt(p) * np.fft.fftn(w)).real
    np.testing.assert_allclose(g.var(), 0.25, rtol=0.6)
    d = g + 0.5 * (g * g - 0.25)
    np.testing.assert_allclose(v, synth.visibilities(d), atol=1e-12)
    assert v[0, h, h] == pytest.approx(d[0].sum())  # U = 0 is the plane sum
