"""Pins of the oracle's ablation functions (the unprotected ABS quantizer
of Sec. 6 / Tables 7-8, and the REL decoder with the host library's exp2 of
Sec. 2.3) against numpy arithmetic and the exact verifier."""
import numpy as np
import pytest

import oracle as O


def _expected_unprotected(x, inv):
    with np.errstate(invalid="ignore", over="ignore"):
        q = x * inv.astype(x.dtype)                 # one IEEE multiply in the data type
        r = np.rint(q)                              # round half to even
        out = ~(np.abs(q) < 2.0 ** 30) | ~(np.abs(r) < 2.0 ** 30)
    bins = np.where(out, 0, np.where(out, 0, r)).astype(np.int64).astype(np.int32)
    return bins, out


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_unprotected_bins_are_rint_of_the_product(dtype):
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(200000) * 10.0 ** rng.uniform(-6, 8, 200000)).astype(dtype)
    x[::1000] = np.nan
    x[1::1000] = np.inf
    eb = 1e-3
    q = O.quantize_unprotected(x, eb)
    bins, out = _expected_unprotected(x, np.array(O.consts("abs", dtype, eb).inv))
    assert np.array_equal(q.bins, bins)
    idx = np.arange(x.size)
    assert np.array_equal(((q.mask[idx >> 5] >> (idx & 31)) & 1).astype(bool), out)
    assert np.array_equal(q.payload.view(np.uint8), x[out].view(np.uint8))


def test_unprotected_differs_from_protected_only_where_the_check_fails():
    rng = np.random.default_rng(2)
    x = rng.uniform(1e4, 2e4, 300000).astype(np.float32)
    eb = 1e-3
    qu, qp = O.quantize_unprotected(x, eb), O.quantize(x, "abs", eb)
    idx = np.arange(x.size)
    mu = ((qu.mask[idx >> 5] >> (idx & 31)) & 1).astype(bool)
    mp = ((qp.mask[idx >> 5] >> (idx & 31)) & 1).astype(bool)
    assert not np.any(mu & ~mp)                     # the check only adds outliers
    assert np.array_equal(qu.bins[~mp], qp.bins[~mp])
    # |x| / eb ~ 1e7: the rounding of 1/(2 eb) and of bin * 2 eb break the bound
    bad_u = O.verify_abs(x, O.dequantize(qu), eb)
    assert bad_u > 0 and O.verify_abs(x, O.dequantize(qp), eb) == 0
    # every violation of the unprotected result is at a value the check rejected
    xr = O.dequantize(qu)
    assert O.verify_abs(x[~mp], xr[~mp], eb) == 0
    assert O.verify_abs(x[mp & ~mu], xr[mp & ~mu], eb) == bad_u


def test_unprotected_equals_protected_for_power_of_two_steps():
    # eb2 = 2^-4: q = x * 16 and bin * eb2 are exact, |x - recon| <= eb2 / 2 = eb
    rng = np.random.default_rng(3)
    x = rng.uniform(-1e5, 1e5, 100000).astype(np.float32)
    eb = 2.0 ** -5
    qu, qp = O.quantize_unprotected(x, eb), O.quantize(x, "abs", eb)
    assert qu.count == qp.count == 0 and np.array_equal(qu.bins, qp.bins)
    assert O.verify_abs(x, O.dequantize(qu), eb) == 0


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_rel_library_recon_against_numpy(dtype):
    rng = np.random.default_rng(4)
    step = float(O.consts("rel", dtype, 1e-3).step)
    b = rng.integers(-60000, 60000, 50000)
    s = rng.integers(0, 2, 50000)
    b[:2], s[:2] = 0, [0, 1]                        # exp2(0) = 1 exactly, with either sign
    bins = (2 * b + s).astype(np.int32)
    mask = np.zeros((bins.size + 31) // 32, np.uint32)
    mask[3] = 0xFFFF0000
    out = O.rel_library_recon(dtype, step, bins, mask)
    assert out[0] == 1.0 and out[1] == -1.0
    assert np.all(out[96 + 16:128] == 0)
    keep = np.ones(bins.size, bool)
    keep[96 + 16:128] = False
    Lr = (b.astype(dtype) * dtype(step)).astype(dtype)
    ref = np.exp2(Lr.astype(np.float64)) if dtype == np.float32 else np.exp2(Lr)
    got = np.abs(out).astype(np.float64)
    ulp = np.spacing(np.abs(ref).astype(dtype)).astype(np.float64)
    # a faithful library exp2 is within one unit in the last place
    assert np.all(np.abs(got[keep] - ref[keep]) <= ulp[keep] * (1.0 if dtype == np.float32 else 2.0))
    assert np.array_equal(np.signbit(out[keep]), s[keep].astype(bool))
