"""Pins of the exact bound verifiers against Python rationals.

The verifiers decide |x - x'| <= eb (Sec. 2.1.1) and
|x|/(1+eps) <= |x'| <= |x|(1+eps) with equal signs (Sec. 2.1.2) without
rounding error.  Here the same decisions are made with fractions.Fraction on
adversarial pairs placed on, just inside and just outside the bound.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O


def _abs_ok(x, y, eb):
    if not (math.isfinite(x) and math.isfinite(y)):
        return np.float64(x).tobytes() == np.float64(y).tobytes()
    return abs(Fraction(x) - Fraction(y)) <= Fraction(eb)


def _rel_ok(x, y, eps):
    if not (math.isfinite(x) and math.isfinite(y)) or x == 0 or y == 0:
        return False
    if math.copysign(1, x) != math.copysign(1, y):
        return False
    a, m, e = abs(Fraction(x)), abs(Fraction(y)), Fraction(eps)
    return a <= m * (1 + e) and m <= a * (1 + e)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_verify_abs_matches_rationals(dtype):
    rng = np.random.default_rng(17)
    xs, ys, ebs = [], [], []
    for _ in range(3000):
        eb = float(10 ** rng.uniform(-8, 2))
        x = dtype(rng.normal(0, 10 ** rng.uniform(-6, 6)))
        d = dtype(eb)
        for y in (x + d, x - d, np.nextafter(x + d, dtype(np.inf)), np.nextafter(x - d, dtype(-np.inf)),
                  np.nextafter(x + d, dtype(-np.inf)), x, dtype(0)):
            xs.append(x); ys.append(dtype(y)); ebs.append(eb)
    xs, ys = np.array(xs, dtype=dtype), np.array(ys, dtype=dtype)
    for k in range(0, len(xs), 7):
        eb = ebs[k]
        sl = slice(k, k + 7)
        want = sum(not _abs_ok(float(a), float(b), eb) for a, b in zip(xs[sl], ys[sl]))
        assert O.verify_abs(xs[sl], ys[sl], eb) == want


def test_verify_abs_half_ulp_case():
    # |x - y| exceeds eb by less than half an ulp of the rounded difference
    eb = 1.0
    x = np.array([2.0], dtype=np.float64)
    y = np.array([1.0 - 2.0 ** -53], dtype=np.float64)   # x - y = 1 + 2^-53 > eb
    assert O.verify_abs(x, y, eb) == 1
    y2 = np.array([1.0], dtype=np.float64)
    assert O.verify_abs(x, y2, eb) == 0


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_verify_rel_matches_rationals(dtype):
    rng = np.random.default_rng(23)
    for _ in range(1500):
        eps = float(10 ** rng.uniform(-7, -0.1))
        x = dtype(rng.choice([-1, 1]) * 10 ** rng.uniform(-30, 30))
        cands = [x * dtype(1 + eps), x / dtype(1 + eps), x * dtype(1 - eps), -x, x, dtype(0),
                 np.nextafter(x * dtype(1 + eps), dtype(np.inf)),
                 np.nextafter(x / dtype(1 + eps), dtype(0))]
        ys = np.array(cands, dtype=dtype)
        xs = np.full(ys.size, x, dtype=dtype)
        want = sum(not (np.array(a).tobytes() == np.array(b).tobytes() or _rel_ok(float(a), float(b), eps))
                   for a, b in zip(xs, ys))
        assert O.verify_rel(xs, ys, eps) == want


def test_verify_flags_non_identical_nan():
    x = np.array([np.nan], dtype=np.float32)
    y = np.array([0x7FC00001], dtype=np.uint32).view(np.float32)
    assert O.verify_abs(x, y, 1.0) == 1
    assert O.verify_abs(x, x.copy(), 1.0) == 0
