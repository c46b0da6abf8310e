"""The split-precision readings checked on the CPU by emulating the operand
formats with numpy (independent of the CUDA kernels): with the power-of-two
field scales of the split-FP16 form no operand overflows FP16, and the
operand rounding of the split forms alone errs by at most ~3 x 2^-22 (FP16)
and ~3 x 2^-17 (BF16, emulated by rounding the FP32 mantissa to 8 bits) of
the sum of |terms|.  The products are summed in FP64 here, so these bound the
operand rounding only; the kernels' FP32 accumulation over K adds the c_acc
term of the error bound, which the GPU error-bound tests cover."""
import numpy as np


def _scale_exp(fmax):
    """k with |F| 2^k < 2^7: 2^(E-1) <= max < 2^E, k = 7 - E (clamped)."""
    if fmax == 0:
        return 0
    E = int(np.frexp(np.float32(fmax))[1])
    return int(np.clip(7 - E, -100, 100))


def _split16(x):
    hi = x.astype(np.float16)
    lo = (x - hi.astype(np.float32)).astype(np.float16)
    return hi, lo


def _bf16(x):
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16  # round to nearest even
    return r.astype(np.uint32).view(np.float32)


def _split_bf16(x):
    hi = _bf16(x)
    return hi, _bf16(x - hi)


def _fields(seed, n, amp):
    r = np.random.default_rng(seed)
    f = r.normal(size=(3, n)).astype(np.float32) * np.float32(amp)
    f[2] *= 1e3  # three fields of different magnitudes
    return f


def test_split_fp16_headroom_and_error_bound():
    for seed, amp in ((1, 1.0), (2, 1e-12), (3, 3e11)):
        fi, fj, fl = _fields(seed, 4096, amp)
        ks = [_scale_exp(np.abs(f).max()) for f in (fi, fj, fl)]
        si, sj, sl = (np.float32(2.0 ** k) for k in ks)
        a_hi, a_lo = _split16(fl * sl)
        assert np.all(np.isfinite(a_hi.astype(np.float32))) and np.abs(fl * sl).max() < 2 ** 7
        p = (fi * np.float32(2.0 ** (ks[0] + ks[1]))) * fj
        assert np.abs(p).max() < 2 ** 14  # FP16 holds 65504
        p_hi, p_lo = _split16(p)
        terms = (a_hi.astype(np.float64) * p_hi + a_hi.astype(np.float64) * p_lo +
                 a_lo.astype(np.float64) * p_hi)
        got = terms.sum() * 2.0 ** -(sum(ks))
        exact = np.sum(fi.astype(np.float64) * fj * fl)
        absum = np.sum(np.abs(fi.astype(np.float64) * fj * fl))
        assert abs(got - exact) <= 3 * 2.0 ** -22 * absum * 1.01, (seed, abs(got - exact) / absum)


def test_split_bf16_error_bound():
    fi, fj, fl = _fields(4, 4096, 1.0)
    a_hi, a_lo = _split_bf16(fl)
    p_hi, p_lo = _split_bf16(fi * fj)
    d = lambda x: x.astype(np.float64)
    got = np.sum(d(a_hi) * d(p_hi) + d(a_hi) * d(p_lo) + d(a_lo) * d(p_hi))
    exact = np.sum(d(fi) * d(fj) * d(fl))
    absum = np.sum(np.abs(d(fi) * d(fj) * d(fl)))
    assert abs(got - exact) <= 3 * 2.0 ** -17 * absum
    # and it is markedly looser than split FP16 on the same data
    ks = [_scale_exp(np.abs(f).max()) for f in (fi, fj, fl)]
    a16h, a16l = _split16(fl * np.float32(2.0 ** ks[2]))
    p16h, p16l = _split16((fi * np.float32(2.0 ** (ks[0] + ks[1]))) * fj)
    got16 = np.sum(d(a16h) * d(p16h) + d(a16h) * d(p16l) + d(a16l) * d(p16h)) * 2.0 ** -sum(ks)
    assert abs(got16 - exact) < abs(got - exact)
