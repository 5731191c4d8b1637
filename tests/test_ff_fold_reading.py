"""Error of the float-float skinny product, restated in NumPy on the CPU.

The CUDA product behind PM_FLAG_FF_CONFIRM works as follows.
  * The operator entry a = a_hi + a_lo is a 24+24-bit split.
  * x = x_hi + x_lo is rounded to nearest.
  * For each term, the FMA-exact error of a_hi x_hi and the first-order
    cross terms a_hi x_lo and a_lo x_hi, gathered by one FMA chain, go to lo.
  * The TwoSum error of hi + a_hi x_hi also goes to lo.
  * (hi, lo) is folded into an FP64 sum every 16 terms.
This restatement checks that the folded sum stays within the bound the
library states, ~9e-13 of sum |a||x|, and that folding is what makes the
difference against one long float-float sum.
"""
from fractions import Fraction

import numpy as np

f32, f64 = np.float32, np.float64


def _trunc24(v):
    m, e = np.frexp(v)
    return np.ldexp(np.trunc(m * 2.0 ** 24) / 2.0 ** 24, e)


def _two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def _ff_dot(ah, al, xh, xl, fold):
    acc, hi, lo = 0.0, f32(0), f32(0)
    for j in range(len(ah)):
        p = f32(ah[j] * xh[j])
        t = f32(f64(ah[j]) * f64(xh[j]) - f64(p))                    # exact product error (FMA)
        t = f32(f64(ah[j]) * f64(xl[j]) + f64(t))                    # FMA chain of the cross terms
        t = f32(f64(al[j]) * f64(xh[j]) + f64(t))
        hi, e = _two_sum(hi, p)
        lo = f32(lo + f32(e + t))
        if fold and (j + 1) % fold == 0:
            acc += f64(hi) + f64(lo)
            hi, lo = f32(0), f32(0)
    return acc + f64(hi) + f64(lo)


def test_folded_float_float_sum_stays_within_the_stated_bound():
    rng = np.random.default_rng(11)
    n = 2048
    worst = {0: 0.0, 16: 0.0}
    for trial in range(6):
        a = rng.standard_normal(n) * np.exp(rng.uniform(-4, 4, n))
        x = rng.standard_normal(n) * np.exp(rng.uniform(-2, 2, n))
        if trial % 2:                       # heavy cancellation: the exact sum nearly vanishes
            a[n // 2:] = -a[: n // 2] * (1 + 1e-9 * rng.standard_normal(n // 2))
            x[n // 2:] = x[: n // 2]
        a_hi = _trunc24(a).astype(f32)
        a_lo = _trunc24(a - a_hi.astype(f64)).astype(f32)
        a_st = a_hi.astype(f64) + a_lo.astype(f64)                   # the stored operator entry
        x_hi = x.astype(f32)
        x_lo = (x - x_hi.astype(f64)).astype(f32)
        exact = float(sum(Fraction(float(u)) * Fraction(float(v)) for u, v in zip(a_st, x)))
        scale = float(np.sum(np.abs(a_st) * np.abs(x)))
        for fold in worst:
            err = abs(_ff_dot(a_hi, a_lo, x_hi, x_lo, fold) - exact) / scale
            worst[fold] = max(worst[fold], err)
    assert worst[16] <= 9e-13
    assert worst[16] < 1e-14 and worst[16] < worst[0]
