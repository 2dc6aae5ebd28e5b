"""Exactly rounded fused multiply-add for the two brute-force executors.

Both the GCN interpreter and the OpenCL evaluator need fma with a single
rounding (v_fma_f32 / v_fma_f64 and OpenCL fma()).  numpy has no fma, so the
exact value a*b+c is formed as a Fraction and rounded to nearest-even.
"""
from fractions import Fraction
import math

import numpy as np


def _round_f32(x: Fraction) -> np.float32:
    if x == 0:
        return np.float32(0.0)
    sign = -1 if x < 0 else 1
    x = abs(x)
    e = x.numerator.bit_length() - x.denominator.bit_length()
    if Fraction(2) ** e > x:
        e -= 1
    elif Fraction(2) ** (e + 1) <= x:
        e += 1
    q = max(e - 23, -149)
    scaled = x / (Fraction(2) ** q)
    m = scaled.numerator // scaled.denominator
    rem = scaled - m
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and m % 2 == 1):
        m += 1
    val = Fraction(m) * Fraction(2) ** q
    if val >= Fraction(2) ** 128:
        return np.float32(sign * np.inf)
    return np.float32(sign * float(val))


def fma32(a, b, c) -> np.float32:
    a, b, c = np.float32(a), np.float32(b), np.float32(c)
    if not (math.isfinite(a) and math.isfinite(b) and math.isfinite(c)):
        with np.errstate(all="ignore"):
            return np.float32(np.float64(a) * np.float64(b) + np.float64(c))
    exact = Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c))
    if exact == 0:
        # sign of an exact zero: -0 only when both addends are -0 (round-to-nearest)
        p = Fraction(float(a)) * Fraction(float(b))
        neg_p = p == 0 and (math.copysign(1, a) * math.copysign(1, b) < 0)
        if neg_p and math.copysign(1, c) < 0:
            return np.float32(-0.0)
        return np.float32(0.0)
    return _round_f32(exact)


def fma64(a, b, c) -> np.float64:
    a, b, c = float(a), float(b), float(c)
    if not (math.isfinite(a) and math.isfinite(b) and math.isfinite(c)):
        with np.errstate(all="ignore"):
            return np.float64(a * b + c)
    exact = Fraction(a) * Fraction(b) + Fraction(c)
    if exact == 0:
        neg_p = (a == 0 or b == 0) and math.copysign(1, a) * math.copysign(1, b) < 0
        if neg_p and math.copysign(1, c) < 0:
            return np.float64(-0.0)
        return np.float64(0.0)
    try:
        return np.float64(exact.numerator / exact.denominator)
    except OverflowError:
        return np.float64(math.copysign(math.inf, exact))
