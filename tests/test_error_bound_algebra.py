"""The two composite error bounds of bs_mabs_error_bound checked as algebra,
independently of the kernels: perturbations of the exact sums within their
per-evaluation bounds (random ones and the worst-case signs) never exceed the
composite bound, and the worst case reaches it.

* General (non-Hermitian) input: S = S(i) of the cubic S(t) is combined from
  the real evaluations at t = 0, 1, -1, 2 as Re S = 2 S(0) - (S(1) + S(-1))/2
  and Im S = (9 S(1) - S(-1) - 2 S(2) - 6 S(0))/6; with |dS(t)| <= b_t the
  bounds are 2 b_0 + (b_1 + b_-1)/2 and (9 b_1 + b_-1 + 2 b_2 + 6 b_0)/6.
* Per-channel sampling: R = S_D / (A S_I) from computed sums S^ = S + dS with
  |dS_D| <= b_D, |dS_I| <= b_I; |R^ - R| <= (b_D / A + |R^| b_I) / (S^_I - b_I)
  for S^_I > b_I (the same with bin means for the ratio-of-sums collapse)."""
import itertools

import numpy as np


def _combine(s0, s1, sm, s2):
    return 2 * s0 - 0.5 * (s1 + sm), (9 * s1 - sm - 2 * s2 - 6 * s0) / 6


def test_combination_recovers_the_cubic_at_i():
    """The four-point combination gives P0 - P2 + i (P1 - P3) for any cubic."""
    r = np.random.default_rng(1)
    for _ in range(100):
        p = r.standard_normal(4)
        S = lambda t: p[0] + p[1] * t + p[2] * t ** 2 + p[3] * t ** 3
        re, im = _combine(S(0), S(1), S(-1), S(2))
        assert abs(re - (p[0] - p[2])) < 1e-12 and abs(im - (p[1] - p[3])) < 1e-12


def test_general_bound_covers_and_is_attained():
    r = np.random.default_rng(2)
    for _ in range(200):
        s = r.standard_normal(4) * 10 ** r.uniform(-3, 3)
        b = np.abs(r.standard_normal(4)) * 10 ** r.uniform(-9, -3)
        bre = 2 * b[0] + 0.5 * (b[1] + b[2])
        bim = (9 * b[1] + b[2] + 2 * b[3] + 6 * b[0]) / 6
        bound = np.hypot(bre, bim)
        re0, im0 = _combine(*s)
        tiny = 1e-14 * np.abs(s).max()  # the FP64 rounding of the combination itself
        worst_re = worst_im = 0.0
        for signs in itertools.product((-1, 1), repeat=4):
            d = np.array(signs) * b
            re, im = _combine(*(s + d))
            worst_re = max(worst_re, abs(re - re0))
            worst_im = max(worst_im, abs(im - im0))
            assert abs(re - re0) <= bre * (1 + 1e-9) + tiny
            assert abs(im - im0) <= bim * (1 + 1e-9) + tiny
            assert np.hypot(re - re0, im - im0) <= bound * (1 + 1e-9) + tiny
        for _ in range(20):  # interior perturbations
            d = r.uniform(-1, 1, 4) * b
            re, im = _combine(*(s + d))
            assert np.hypot(re - re0, im - im0) <= bound * (1 + 1e-9) + tiny
        # each part's bound is reached by its own worst signs
        np.testing.assert_allclose(worst_re, bre, rtol=1e-6, atol=tiny)
        np.testing.assert_allclose(worst_im, bim, rtol=1e-6, atol=tiny)


def _ratio_bound(sd_hat, si_hat, bd, bi, A):
    R_hat = sd_hat / (A * si_hat)
    den = si_hat - bi
    return (bd / A + abs(R_hat) * bi) / den if den > 0 else np.inf


def test_ratio_bound_covers_and_is_attained():
    r = np.random.default_rng(3)
    for _ in range(500):
        A = 10 ** r.uniform(-1, 1)
        sd = r.standard_normal() * 10 ** r.uniform(-2, 4)
        si = 10 ** r.uniform(0, 6)  # a denominator: a positive sum of occupancies
        bd = abs(sd) * 10 ** r.uniform(-7, -2) + 1e-12
        bi = si * 10 ** r.uniform(-7, -1)
        R = sd / (A * si)
        worst, worst_bound = 0.0, None
        for ed, ei in itertools.product((-1, 1), repeat=2):
            sdh, sih = sd + ed * bd, si + ei * bi
            e = abs(sdh / (A * sih) - R)
            bound = _ratio_bound(sdh, sih, bd, bi, A)
            assert e <= bound * (1 + 1e-9)
            if e > worst:
                worst, worst_bound = e, bound
        for _ in range(20):
            sdh, sih = sd + r.uniform(-1, 1) * bd, si + r.uniform(-1, 1) * bi
            assert abs(sdh / (A * sih) - R) <= _ratio_bound(sdh, sih, bd, bi, A) * (1 + 1e-9)
        # the bound is tight to first order: at the worst signs it exceeds the
        # error only by terms of relative size b_I / S_I (it uses R^ and S^_I - b_I)
        assert worst >= worst_bound * (1 - 4 * bi / si) - 1e-15 * abs(R)


def test_ratio_of_sums_bound_from_bin_means():
    """The collapse sums K channel triples: with per-triple bounds b_D, b_I the
    sums' errors are at most K b_D and K b_I, and the bin-mean form
    (b_D/A + |R^| b_I) / (<S^_I> - b_I) equals the bound of the sums."""
    r = np.random.default_rng(4)
    for _ in range(200):
        K = int(r.integers(1, 50))
        A = 1.7
        sd = r.standard_normal(K) * 100
        si = 10 ** r.uniform(1, 4, K)
        bd, bi = 1e-3, 1e-2
        d_d, d_i = r.uniform(-1, 1, K) * bd, r.uniform(-1, 1, K) * bi
        R = sd.sum() / (A * si.sum())
        sdh, sih = (sd + d_d).sum(), (si + d_i).sum()
        Rh = sdh / (A * sih)
        mean_form = (bd / A + abs(Rh) * bi) / (sih / K - bi)
        sum_form = _ratio_bound(sdh, sih, K * bd, K * bi, A)
        np.testing.assert_allclose(mean_form, sum_form, rtol=1e-12)
        assert abs(Rh - R) <= mean_form * (1 + 1e-9)
