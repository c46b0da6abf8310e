"""CPU tests of the register FFT (csrc/fft_reg.cuh) and of the exact
FP32 <-> FP64 conversions (csrc/fp_bits.cuh), compiled as host code with nvcc
through tests/host_fft_reg.cu.  The DFTs are checked against numpy's FFT (the
DFT definition, to FP32 rounding: normwise error below 8 u log2 N), the
conversions bit for bit against numpy's IEEE conversions, including
rounding ties, subnormals, overflow, zeros, infinities and NaNs."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2506_10526_gb300", "csrc")
U = 2.0 ** -24


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = tmp_path_factory.mktemp("freg") / "host_fft_reg"
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-I", CSRC, "-o", str(out),
                        os.path.join(HERE, "host_fft_reg.cu")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return str(out)


def _call(driver, tmp_path, args, x, out_dtype):
    src, dst = tmp_path / "in.bin", tmp_path / "out.bin"
    np.ascontiguousarray(x).tofile(src)
    r = subprocess.run([driver, *[str(a) for a in args], str(src), str(dst)],
                       capture_output=True, text=True)
    assert r.returncode == 0, (args, r.returncode, r.stderr)
    return np.fromfile(dst, dtype=out_dtype)


def _ref_dft(x, sign):
    # sign -1: numpy's forward DFT; +1: the unnormalised inverse
    return np.fft.fft(x, axis=-1) if sign < 0 else np.fft.ifft(x, axis=-1) * x.shape[-1]


@pytest.mark.parametrize("mode,lengths", [("dft", [2, 3, 4, 5, 6, 8, 9, 10, 12, 15, 16, 18, 20,
                                                   24, 25, 27, 30, 32]),
                                          ("fft2", [16, 24, 32, 48, 64, 96, 128, 192, 256,
                                                    384, 512, 768, 540, 675, 729, 750])])
@pytest.mark.parametrize("sign", [1, -1])
def test_register_dft_against_numpy(driver, tmp_path, mode, lengths, sign):
    rng = np.random.default_rng(7)
    for L in lengths:
        x = (rng.normal(size=(6, L)) + 1j * rng.normal(size=(6, L))).astype(np.complex64)
        x[0] = 0
        x[1] = 0
        x[1, 0] = 1  # impulse: a flat spectrum
        x[2] = np.exp(2j * np.pi * 3 * np.arange(L) / L)  # one frequency
        got = _call(driver, tmp_path, [mode, L, sign], x, np.complex64).reshape(x.shape)
        ref = _ref_dft(x.astype(np.complex128), sign)
        err = np.linalg.norm(got - ref, axis=-1) / np.maximum(np.linalg.norm(ref, axis=-1), 1e-300)
        bound = 8 * U * np.log2(L) + 4 * U
        assert np.all(got[0] == 0), (L, "zero input")
        assert err[1:].max() < bound, (mode, L, sign, err.max(), bound)
        # the single frequency lands in one bin
        k = 3 % L if sign < 0 else (-3) % L
        assert np.argmax(np.abs(got[2])) == k


def test_f64_to_f32_bit_exact(driver, tmp_path):
    rng = np.random.default_rng(11)
    bits = rng.integers(0, 2 ** 63, size=400000, dtype=np.int64).astype(np.uint64)
    bits[::2] |= np.uint64(1 << 63)
    x = bits.view(np.float64)
    # values on and next to FP32 rounding ties, subnormals and the overflow edge
    f = rng.normal(size=20000).astype(np.float32) * np.float32(1e3)
    d = f.astype(np.float64).view(np.uint64)
    ties = np.concatenate([d + np.uint64(1 << 28), d - np.uint64(1 << 28), d + np.uint64(1),
                           d + np.uint64((1 << 28) + 1)]).view(np.float64)
    small = np.ldexp(rng.uniform(0.5, 1.0, 20000), rng.integers(-152, -120, 20000))
    edge = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 3.4028235677973366e38,
                     3.4028235677973362e38, 3.402823669209385e38, 1.401298464324817e-45,
                     7.006492321624085e-46, 7.006492321624087e-46, 1e-320, -1e-320, 1e300])
    x = np.concatenate([x, ties, small, -small, edge])
    with np.errstate(all="ignore"):
        ref = x.astype(np.float32)
    got = _call(driver, tmp_path, ["d2f"], x, np.float32)
    same = (got.view(np.uint32) == ref.view(np.uint32)) | (np.isnan(got) & np.isnan(ref))
    assert same.all(), x[~same][:5]


@pytest.mark.parametrize("e2", [0, 1, -7, 49, -60])
def test_f32_to_f64_scaled_bit_exact(driver, tmp_path, e2):
    rng = np.random.default_rng(100 + e2)
    f = rng.integers(0, 2 ** 32, size=300000, dtype=np.uint64).astype(np.uint32).view(np.float32)
    f = np.concatenate([f, np.array([0.0, -0.0, np.inf, -np.inf, 1e-45, -3e-39, 1.1754942e-38],
                                    np.float32)])
    got = _call(driver, tmp_path, ["f2d", e2], f, np.float64)
    with np.errstate(all="ignore"):
        ref = np.ldexp(f.astype(np.float64), e2)
    same = (got.view(np.uint64) == ref.view(np.uint64)) | (np.isnan(got) & np.isnan(ref))
    assert same.all(), f[~same][:5]
