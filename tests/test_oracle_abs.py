"""Pins of the oracle's ABS quantizer (Sec. 2.1.1, 2.2, 3.1, 3.3).

Independent references used here:
  * power-of-two bounds, where x / (2 eb) is exact, so the bins must equal
    numpy.rint of the exact product and every finite value with |q| < 2^30 is
    quantizable (|x - bin 2eb| <= eb holds exactly);
  * the exact-arithmetic verifier (itself pinned in test_oracle_verifier.py);
  * numpy bit packing for the outlier mask and payload layout.
"""
import numpy as np
import pytest

import oracle as O


def _mask_words(flags):
    n = flags.size
    w = (n + 31) // 32
    f = np.zeros(w * 32, dtype=np.uint64)
    f[:n] = flags
    return (f.reshape(w, 32) << np.arange(32, dtype=np.uint64)).sum(axis=1).astype(np.uint32)


def _mixed_f32(rng, n):
    mags = 10.0 ** rng.uniform(-12, 8, n)
    x = (mags * rng.choice([-1.0, 1.0], n)).astype(np.float32)
    return x


@pytest.mark.parametrize("dtype,k", [(np.float32, 10), (np.float32, 3), (np.float64, 20),
                                     (np.float64, 7)])
def test_power_of_two_bound_closed_form(dtype, k):
    eb = 2.0 ** -k
    rng = np.random.default_rng(k)
    n = 20000
    x = np.concatenate([
        _mixed_f32(rng, n).astype(dtype),
        # ties q = j + 1/2 (x exactly on a bin edge): RNE picks the even bin,
        # and |x - recon| == eb must be accepted (the paper's "> eb" test)
        ((rng.integers(-5000, 5000, 2000) + 0.5) * 2 * eb).astype(dtype),
        # the maxbin edge and the INT_MIN edge (Sec. 2.4, 3.3)
        np.array([(2.0 ** 30 - 64) * 2 * eb, 2.0 ** 30 * 2 * eb, -(2.0 ** 30) * 2 * eb,
                  -(2.0 ** 31) * 2 * eb, (2.0 ** 31) * 2 * eb, -(2.0 ** 30 - 64) * 2 * eb],
                 dtype=dtype),
    ])
    q = O.quantize(x, "abs", eb)
    c = q.consts
    assert c.ebT == eb and c.eb2 == 2 * eb and c.inv == 1 / (2 * eb)
    qd = x.astype(np.float64) / (2 * eb)  # exact: division by a power of two
    expect_out = ~(np.abs(qd) < 2.0 ** 30)
    flags = np.zeros(x.size, dtype=bool)
    flags[:] = ((q.mask[np.arange(x.size) >> 5] >> (np.arange(x.size) & 31)) & 1).astype(bool)
    assert np.array_equal(flags, expect_out)
    want_bins = np.where(expect_out, 0, np.rint(np.where(expect_out, 0, qd))).astype(np.int32)
    assert np.array_equal(q.bins, want_bins)
    # on ties the even neighbour is chosen
    ties = np.abs(qd - np.floor(qd) - 0.5) == 0
    assert np.all(q.bins[ties & ~expect_out] % 2 == 0)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("eb", [1e-2, 1e-3, 1e-4, 1e-5, 0.3, 7.0])
def test_bound_holds_exactly(dtype, eb):
    rng = np.random.default_rng(int(eb * 1e6) + 7)
    n = 50000
    i = np.arange(n)
    x = np.concatenate([
        (np.sin(0.001 * i) * 100 + rng.normal(0, 0.1, n)).astype(dtype),
        _mixed_f32(rng, n).astype(dtype),
        (rng.integers(-10 ** 6, 10 ** 6, n) * (2 * eb) * (1 + rng.uniform(-1e-7, 1e-7, n))).astype(dtype),
    ])
    q = O.quantize(x, "abs", eb)
    xr = O.dequantize(q)
    assert O.verify_abs(x, xr, eb) == 0
    idx = np.arange(x.size)
    out = ((q.mask[idx >> 5] >> (idx & 31)) & 1).astype(bool)
    ub = np.uint32 if dtype == np.float32 else np.uint64
    assert np.array_equal(xr.view(ub)[out], x.view(ub)[out])
    assert np.all(q.bins[out] == 0)
    # decoded inliers are bin * eb2 as one IEEE multiplication
    eb2 = dtype(q.consts.eb2)
    assert np.array_equal(xr[~out].view(ub), (q.bins[~out].astype(dtype) * eb2).view(ub))


def test_smooth_data_outlier_rate_is_small():
    # Rounding failures are rare on smooth data (Table 9: averages 0.00-3.41%)
    rng = np.random.default_rng(11)
    i = np.arange(1 << 18)
    x = (np.sin(0.001 * i) * 100 + rng.normal(0, 0.1, i.size)).astype(np.float32)
    q = O.quantize(x, "abs", 1e-3)
    assert q.count < 0.01 * x.size


def test_special_values_f32():
    f = np.float32
    specials = np.array([0x7FC00000, 0x7F800001, 0xFFC01234, 0x7FBFFFFF,  # NaNs
                         0x7F800000, 0xFF800000,                          # +/-Inf
                         0x00000000, 0x80000000,                          # +/-0
                         0x00000001, 0x807FFFFF, 0x00400000,              # denormals
                         0x7F7FFFFF, 0xFF7FFFFF,                          # +/-FLT_MAX
                         0x00800000], dtype=np.uint32).view(f)            # FLT_MIN
    q = O.quantize(specials, "abs", 1e-3)
    xr = O.dequantize(q)
    flags = [(q.mask[0] >> i) & 1 for i in range(specials.size)]
    assert flags == [1, 1, 1, 1, 1, 1, 0, 0, 0, 0, 0, 1, 1, 0]
    # outliers are kept bit for bit, payload in index order
    assert list(q.payload) == list(specials.view(np.uint32)[[0, 1, 2, 3, 4, 5, 11, 12]])
    # +/-0 and denormals sit in bin 0 and decode as +0 (reading R7; Sec. 3.1:
    # denormals are treated like normal values)
    assert np.all(q.bins[6:11] == 0) and np.all(xr[6:11].view(np.uint32) == 0)
    assert O.verify_abs(specials, xr, 1e-3) == 0


def test_special_values_f64():
    specials = np.array([0x7FF8000000000000, 0x7FF0000000000001, 0xFFF8000000000123,
                         0x7FF0000000000000, 0xFFF0000000000000, 0, 0x8000000000000000,
                         1, 0x800FFFFFFFFFFFFF, 0x7FEFFFFFFFFFFFFF], dtype=np.uint64).view(np.float64)
    q = O.quantize(specials, "abs", 1e-3)
    xr = O.dequantize(q)
    flags = [(q.mask[0] >> i) & 1 for i in range(specials.size)]
    assert flags == [1, 1, 1, 1, 1, 0, 0, 0, 0, 1]
    assert np.array_equal(xr.view(np.uint64)[[0, 1, 2, 3, 4, 9]],
                          specials.view(np.uint64)[[0, 1, 2, 3, 4, 9]])
    assert O.verify_abs(specials, xr, 1e-3) == 0


@pytest.mark.parametrize("n", [1, 31, 32, 33, 1000, 4097])
def test_mask_and_payload_layout(n):
    rng = np.random.default_rng(n)
    x = rng.normal(0, 1, n).astype(np.float32)
    idx = np.sort(rng.choice(n, size=max(1, n // 10), replace=False))
    bits = x.view(np.uint32).copy()
    bits[idx] = 0x7FC00000 | rng.integers(0, 1 << 22, idx.size).astype(np.uint32)
    x = bits.view(np.float32)
    # power-of-two bound so that no rounding failure adds outliers
    q = O.quantize(x, "abs", 2.0 ** -12)
    flags = np.zeros(n, dtype=np.uint64)
    flags[idx] = 1
    assert np.array_equal(q.mask, _mask_words(flags))
    assert q.count == idx.size
    assert np.array_equal(q.payload, bits[idx])
    assert np.all(q.bins[idx] == 0)


def test_capacity_truncates_payload_but_counts_all():
    x = np.full(100, np.nan, dtype=np.float32)
    q = O.quantize(x, "abs", 1e-3, capacity=10)
    assert q.count == 100 and q.payload.size == 10


def test_empty_input():
    x = np.zeros(0, dtype=np.float32)
    q = O.quantize(x, "abs", 1e-3)
    assert q.count == 0 and q.bins.size == 0 and q.mask.size == 0


@pytest.mark.parametrize("eb", [0.0, -1.0, float("nan"), float("inf"), 1e-46, 1e39])
def test_bad_bounds_rejected_f32(eb):
    with pytest.raises(O.BoundError):
        O.consts("abs", np.float32, eb)


def test_ebT_is_rounded_down():
    from fractions import Fraction
    for eb in (1e-3, 1e-5, 0.1, 3.3, 1e-30):
        c = O.consts("abs", np.float32, eb)
        e = np.float32(c.ebT)
        assert Fraction(float(e)) <= Fraction(eb)
        assert Fraction(float(np.nextafter(e, np.float32(np.inf)))) > Fraction(eb)
        assert c.eb2 == 2 * c.ebT
        # inv is the correctly rounded float reciprocal of eb2
        r = Fraction(1) / Fraction(c.eb2)
        inv = np.float32(c.inv)
        lo, hi = np.nextafter(inv, np.float32(0)), np.nextafter(inv, np.float32(np.inf))
        assert abs(Fraction(float(inv)) - r) <= abs(Fraction(float(lo)) - r)
        assert abs(Fraction(float(inv)) - r) <= abs(Fraction(float(hi)) - r)
