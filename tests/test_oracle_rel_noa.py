"""Pins of the oracle's REL (Sec. 2.1.2, 3.2) and NOA (Sec. 2.1.3) quantizers.

REL: the bound is checked exactly on every element; the decoder is checked
against the closed form of pow2approx; the bin choice is checked to be the
nearest log-domain bin; the acceptance constant is checked to keep one
rounding inside the bound; special values are outliers (reading R4).
NOA: the range and the derived absolute bound are checked against exact
rational arithmetic with rounding toward -infinity (reading R6).
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O


def _flags(q, n):
    idx = np.arange(n)
    return ((q.mask[idx >> 5] >> (idx & 31)) & 1).astype(bool)


def _mags(rng, n, lo, hi, dtype):
    x = 10.0 ** rng.uniform(lo, hi, n) * rng.choice([-1.0, 1.0], n)
    return x.astype(dtype)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("eps", [1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6])
def test_rel_bound_holds_exactly(dtype, eps):
    rng = np.random.default_rng(int(-math.log10(eps)) + (0 if dtype == np.float32 else 50))
    lo, hi = (-37, 38) if dtype == np.float32 else (-300, 300)
    x = np.concatenate([_mags(rng, 60000, lo, hi, dtype), _mags(rng, 20000, -3, 3, dtype)])
    q = O.quantize(x, "rel", eps)
    xr = O.dequantize(q)
    assert O.verify_rel(x, xr, eps) == 0
    out = _flags(q, x.size)
    # sign folded into the stored bin (reading R4)
    assert np.array_equal((q.bins[~out] & 1).astype(bool), np.signbit(x[~out]))


def test_rel_specials_are_outliers():
    bits = np.array([0x00000000, 0x80000000, 0x00000001, 0x807FFFFF, 0x7F800000, 0xFF800000,
                     0x7FC00000, 0xFFC00001, 0x3F800000, 0xBF800000], dtype=np.uint32)
    x = bits.view(np.float32)
    q = O.quantize(x, "rel", 1e-3)
    f = _flags(q, x.size)
    assert list(f) == [True] * 8 + [False, False]
    assert np.array_equal(q.payload, bits[:8])
    xr = O.dequantize(q)
    assert xr[8] == 1.0 or abs(xr[8] - 1.0) <= 1e-3
    assert xr[9] < 0


@pytest.mark.parametrize("eps", [1e-2, 1e-3, 1e-4])
def test_rel_decode_matches_pow2_closed_form(eps):
    rng = np.random.default_rng(99)
    x = _mags(rng, 20000, -30, 30, np.float32)
    q = O.quantize(x, "rel", eps)
    out = _flags(q, x.size)
    xr = O.dequantize(q)
    b = (q.bins[~out] >> 1).astype(np.float32)  # arithmetic shift: b = (bin - s)/2
    s = (q.bins[~out] & 1).astype(bool)
    Lr = b * np.float32(q.consts.step)                      # one float multiplication
    bb = (Lr + np.float32(127.0)).astype(np.float64)        # one float addition
    k = np.floor(bb)
    m = np.ldexp(1.0 + (bb - k), (k - 127).astype(np.int64)).astype(np.float32)
    want = np.where(s, -m, m).astype(np.float32)
    assert np.array_equal(xr[~out].view(np.uint32), want.view(np.uint32))


def test_rel_bin_is_nearest_log_domain_bin():
    # b must be the integer nearest to L / step (rint, not floor or trunc).
    rng = np.random.default_rng(5)
    x = _mags(rng, 5000, -5, 5, np.float32)
    eps = 1e-3
    q = O.quantize(x, "rel", eps)
    out = _flags(q, x.size)
    step = Fraction(q.consts.step)
    inv = Fraction(q.consts.inv_l)
    for xi, bi in zip(x[~out][:2000], q.bins[~out][:2000]):
        L = Fraction(float(O.log2approx_f32(abs(float(xi)))))
        b = int(bi) >> 1
        # q = RN(L * inv_l) is within half an ulp of the exact product; the
        # chosen bin is within 1/2 (+ that rounding) of L / step
        assert abs(L * inv - b) <= Fraction(1, 2) + Fraction(1, 1 << 20)
        assert abs(L / step - b) <= Fraction(1, 2) + Fraction(1, 1 << 10)


def test_rel_outlier_rate_moderate_exponents():
    # where the log domain has far more resolution than the step, only edge
    # cases of the piecewise-linear approximation may fail
    rng = np.random.default_rng(8)
    x = _mags(rng, 100000, -4, 4, np.float32)
    q = O.quantize(x, "rel", 1e-3)
    assert q.count < 0.01 * x.size


@pytest.mark.parametrize("dtype,p", [(np.float32, 23), (np.float64, 52)])
@pytest.mark.parametrize("eps", [1e-1, 1e-3, 1e-6, 0.999])
def test_rel_constants(dtype, p, eps):
    c = O.consts("rel", dtype, eps)
    eT = Fraction(c.ebT)
    assert eT <= Fraction(eps)
    if dtype == np.float32:
        assert Fraction(float(np.nextafter(np.float32(c.ebT), np.float32(1)))) > Fraction(eps)
    # one round-to-nearest of y * chk stays within y * e_T (for normal results)
    assert Fraction(c.chk) * (1 + Fraction(1, 1 << (p + 1))) <= eT
    # the log-domain half step is eb/(1+eb) up to a few roundings
    target = eT / (1 + eT)
    assert abs(Fraction(c.lb) - target) <= target * Fraction(4, 1 << p)
    assert Fraction(c.step) == 2 * Fraction(c.lb)
    r = 1 / Fraction(c.step)
    assert abs(Fraction(c.inv_l) - r) <= r * Fraction(1, 1 << (p + 1))


# ---------------------------------------------------------------- NOA ----

def _rd(fr):
    """Largest double <= the rational fr."""
    d = float(fr)
    if Fraction(d) > fr:
        d = math.nextafter(d, -math.inf)
    return d


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_noa_range_and_bound_are_rounded_down(dtype):
    rng = np.random.default_rng(3)
    for trial in range(50):
        a, b = rng.uniform(-1e6, 1e6, 2)
        mn, mx = min(a, b), max(a, b)
        x = rng.uniform(mn, mx, 1000).astype(dtype)
        x[rng.integers(0, 1000)] = dtype(mn)
        x[rng.integers(0, 1000)] = dtype(mx)
        x[rng.integers(0, 1000, 5)] = np.nan
        x[rng.integers(0, 1000)] = np.inf
        x[rng.integers(0, 1000)] = -np.inf
        fin = x[np.isfinite(x)]
        eps = float(10 ** rng.uniform(-5, -1))
        c = O.consts("noa", dtype, eps, x=x)
        Rex = Fraction(float(fin.max())) - Fraction(float(fin.min()))
        assert c.R == _rd(Rex)
        assert c.eb_abs == _rd(Fraction(eps) * Fraction(c.R))
        assert Fraction(c.eb_abs) <= Fraction(eps) * Rex
        q = O.quantize_with(c, x)
        xr = O.dequantize(q)
        assert O.verify_abs(x, xr, c.eb_abs) == 0
        # NOA is ABS with the derived bound (Sec. 2.1.3)
        qa = O.quantize_with(O.consts("abs", dtype, c.eb_abs), x)
        assert np.array_equal(qa.bins, q.bins) and np.array_equal(qa.mask, q.mask)


def test_noa_closed_form_two_values():
    x = np.array([-3.0, 5.0, 1.0, np.nan], dtype=np.float64)
    c = O.consts("noa", np.float64, 1e-3, x=x)
    assert c.R == 8.0 and c.eb_abs == _rd(Fraction(1e-3) * 8)


def test_noa_rounding_direction_on_inexact_range():
    # max - min not representable: R must be the double just below
    x = np.array([1.0, -2.0 ** -60], dtype=np.float64)
    c = O.consts("noa", np.float64, 0.5, x=x)
    assert c.R == 1.0
    x = np.array([1.0, 2.0 ** -60], dtype=np.float64)
    c = O.consts("noa", np.float64, 0.5, x=x)
    assert c.R == math.nextafter(1.0, 0.0)


@pytest.mark.parametrize("x", [
    np.array([np.nan, np.inf, -np.inf], dtype=np.float32),   # no finite value
    np.full(77, 3.25, dtype=np.float32),                        # R = 0
    np.array([1.0], dtype=np.float32),                          # one value
])
def test_noa_degenerate_range_stores_everything(x):
    q = O.quantize(x, "noa", 1e-3)
    assert q.consts.all_outliers == 1
    assert q.count == x.size
    assert np.array_equal(q.payload, x.view(np.uint32))
    assert np.array_equal(O.dequantize(q).view(np.uint32), x.view(np.uint32))


def test_noa_tiny_range_f32_falls_back_to_lossless():
    # eps * R below the smallest normal float: every value is stored losslessly
    x = np.array([1.0, np.nextafter(np.float32(1.0), np.float32(2.0))], dtype=np.float32)
    q = O.quantize(x, "noa", 1e-35)
    assert q.consts.all_outliers == 1 and q.count == 2


@pytest.mark.parametrize("x", [
    np.full(9, 3.25, dtype=np.float32),
    np.array([-2.5, -2.5], dtype=np.float64),
    np.array([-0.0, 0.0, -0.0], dtype=np.float32),
    np.array([0.0, -0.0], dtype=np.float64),
    np.array([np.nan, -0.0], dtype=np.float32),
])
def test_noa_zero_range_is_positive_zero(x):
    # R is a length: every zero range is +0 (x - x rounded toward -inf would
    # give -0), whatever signed zeros the data holds and in whatever order
    c = O.consts("noa", x.dtype, 1e-3, x=x)
    assert np.float64(c.R).tobytes() == np.float64(0.0).tobytes()
    assert np.float64(c.eb_abs).tobytes() == np.float64(0.0).tobytes()
    assert c.all_outliers == 1
