"""Pins of the oracle's 16-bit formats (reading R11: binary16 and bfloat16
inputs take the float32 recipe on their exact float value, and the check of
Sec. 3.1 tests the decoder's 16-bit output).

What pins them, independently of the oracle's own arithmetic:
  - widening and round-to-nearest-even against numpy's float16 and torch's
    bfloat16 conversions, over every 16-bit pattern, every midpoint between
    neighbouring 16-bit values and its float32 neighbours, and a stride of all
    float32 patterns;
  - the bound of Sec. 2.1 checked exactly on every 16-bit pattern for several
    bounds (ABS, REL, NOA);
  - ABS with a power-of-two eb2, where every step is exact and the bins,
    outliers and decoded values follow from numpy's rint and float16 casts;
  - REL bins equal the float32 recipe's bins of the widened values wherever
    both accept, and decoding equals the float32 decoding rounded by the
    library conversion;
  - NOA ranges of constructed arrays in closed form.
"""
import numpy as np
import pytest
import torch

import oracle as O

ALL16 = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)


def _bf16_to_f32_lib(h):
    return torch.from_numpy(h.view(np.int16).copy()).view(torch.bfloat16).float().numpy()


def _f32_to_bf16_lib(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16) \
        .view(torch.int16).numpy().view(np.uint16)


def _widen_lib(h, fmt):
    return h.view(np.float16).astype(np.float32) if fmt == "f16" else _bf16_to_f32_lib(h)


def _round_lib(x, fmt):
    x = np.ascontiguousarray(x, dtype=np.float32)
    if fmt == "f16":
        with np.errstate(over="ignore"):
            return x.astype(np.float16).view(np.uint16)
    return _f32_to_bf16_lib(x)


def _as_input(h, fmt):
    return h.view(np.float16) if fmt == "f16" else h


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_widen_matches_library_on_every_pattern(fmt):
    w = O.widen16(ALL16, fmt)
    ref = _widen_lib(ALL16, fmt)
    assert np.array_equal(w.view(np.uint32), ref.view(np.uint32))


def _boundary_floats(fmt):
    """Every positive and negative midpoint between neighbouring finite
    16-bit values (exact in float32), with its two float32 neighbours."""
    h = ALL16[(ALL16 & 0x7FFF) < (0x7C00 if fmt == "f16" else 0x7F80)]
    v = O.widen16(h, fmt).astype(np.float64)
    nxt = O.widen16((h + 1).astype(np.uint16), fmt).astype(np.float64)
    pos = h < 0x8000
    mid = ((v + nxt) / 2)[pos].astype(np.float32)  # exact
    assert np.all(mid.astype(np.float64) == ((v + nxt) / 2)[pos])
    m = np.concatenate([mid, -mid, v.astype(np.float32)])
    up = np.nextafter(m, np.float32(np.inf))
    dn = np.nextafter(m, np.float32(-np.inf))
    return np.concatenate([m, up, dn])


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_round_matches_library_at_every_midpoint(fmt):
    x = _boundary_floats(fmt)
    x = x[~np.isnan(x)]
    assert np.array_equal(O.round16(x, fmt), _round_lib(x, fmt))


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_round_matches_library_on_strided_float32(fmt):
    u = np.arange(0, 1 << 32, 1021, dtype=np.uint64).astype(np.uint32)
    x = u.view(np.float32)
    x = x[~np.isnan(x)]
    specials = np.array([0.0, -0.0, np.inf, -np.inf, 65504.0, 65519.996, 65520.0, 65536.0,
                         2.0 ** -24, 2.0 ** -25, 2.0 ** -25 * 1.0000001, 3.4e38, -3.4e38,
                         np.finfo(np.float32).tiny, np.finfo(np.float32).tiny / 3], dtype=np.float32)
    x = np.concatenate([x, specials])
    assert np.array_equal(O.round16(x, fmt), _round_lib(x, fmt))


EBS = [1e-1, 1e-2, 1e-3, 3e-4, 1e-5, 1e-8]


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("bound", ["abs", "rel", "noa"])
@pytest.mark.parametrize("eb", EBS)
def test_bound_holds_on_every_pattern(fmt, bound, eb):
    x = _as_input(ALL16, fmt)
    f = None if fmt == "f16" else "bf16"
    q = O.quantize(x, bound, eb, fmt=f)
    xr = O.dequantize(q)
    xr_in = xr if fmt == "f16" else xr.view(np.uint16)
    if bound == "rel":
        assert O.verify_rel(x, xr_in, eb, fmt=f) == 0
    else:
        e = eb if bound == "abs" else q.consts.eb_abs
        assert O.verify_abs(x, xr_in, e, fmt=f) == 0
    # outliers decode to their own bit patterns, in index order
    bits = xr.view(np.uint16)
    idx = np.nonzero((q.mask[np.arange(x.size) >> 5] >> (np.arange(x.size) & 31)) & 1)[0]
    assert idx.size == q.count
    assert np.array_equal(bits[idx], ALL16[idx])
    assert np.array_equal(q.payload, ALL16[idx])
    assert np.all(q.bins[idx] == 0)


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("k", [1, 4, 9, 14])
def test_abs_power_of_two_closed_form(fmt, k):
    """eb = 2^-k: eb2 = 2^(1-k), inv = 2^(k-1), so q = x 2^(k-1) and the
    reconstruction b 2^(1-k) are exact; the bin is numpy's rint of the exact
    quotient and the decoded value numpy's / torch's rounding of the exact
    reconstruction.  An in-range value is an outlier iff that decoded value is
    more than eb away (exact in float64 for 16-bit values)."""
    eb = 2.0 ** -k
    x = _as_input(ALL16, fmt)
    f = None if fmt == "f16" else "bf16"
    q = O.quantize(x, "abs", eb, fmt=f)
    with np.errstate(invalid="ignore"):
        xv = _widen_lib(ALL16, fmt).astype(np.float64)
    fin = np.isfinite(xv)
    qv = np.where(fin, xv * 2.0 ** (k - 1), np.inf)
    inr = np.abs(qv) < 2.0 ** 30
    b = np.where(inr, np.rint(np.where(inr, qv, 0.0)), 0.0)
    inr &= np.abs(b) < 2.0 ** 30
    b = b + 0.0  # integer bins: rint's -0 is the bin 0
    recon = (b * 2.0 ** (1 - k)).astype(np.float32)  # exact
    dec = _widen_lib(_round_lib(recon, fmt), fmt).astype(np.float64)
    with np.errstate(invalid="ignore"):
        ok = inr & (np.abs(xv - dec) <= eb)
    out = (q.mask[np.arange(x.size) >> 5] >> (np.arange(x.size) & 31)) & 1
    assert np.array_equal(out == 0, ok)
    assert np.array_equal(q.bins[ok], b[ok].astype(np.int32))
    xr = O.dequantize(q).view(np.uint16)
    assert np.array_equal(xr[ok], _round_lib(recon[ok], fmt))


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("eb", [1e-2, 1e-3, 1e-5])
def test_rel_bins_and_decoding_follow_the_float32_recipe(fmt, eb):
    x = _as_input(ALL16, fmt)
    f = None if fmt == "f16" else "bf16"
    q16 = O.quantize(x, "rel", eb, fmt=f)
    w = O.widen16(ALL16, fmt)
    q32 = O.quantize(w, "rel", eb)
    n = x.size
    out16 = ((q16.mask[np.arange(n) >> 5] >> (np.arange(n) & 31)) & 1) == 1
    out32 = ((q32.mask[np.arange(n) >> 5] >> (np.arange(n) & 31)) & 1) == 1
    both = ~out16 & ~out32
    assert both.sum() > 0.5 * n
    assert np.array_equal(q16.bins[both], q32.bins[both])
    # decoding: the float32 decoding of the same bins, rounded by the library
    c32 = O.consts("rel", np.float32, eb)
    q32b = O.Quantized(q16.bins, np.zeros_like(q16.mask), np.zeros(0, np.uint32), 0, c32)
    d32 = O.dequantize(q32b)
    d16 = O.dequantize(q16).view(np.uint16)
    assert np.array_equal(d16[~out16], _round_lib(d32[~out16], fmt))
    # float32 zeros, denormals, Inf and NaN are outliers; f16 subnormals are not
    ex = (w.view(np.uint32) >> 23) & 0xFF
    assert np.all(out16[(ex == 0) | (ex == 0xFF)])
    if fmt == "f16" and eb >= 1e-2:
        sub = ((ALL16 & 0x7C00) == 0) & ((ALL16 & 0x3FF) != 0)
        assert (~out16[sub]).sum() > 0


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_noa_range_closed_form(fmt):
    rng = np.random.default_rng(3)
    for _ in range(50):
        a, b = rng.uniform(-100, 100, 2)
        vals = np.array([a, b, (a + b) / 2, np.inf, -np.inf, np.nan], dtype=np.float32)
        h = _round_lib(vals[:3], fmt)
        specials = _round_lib(np.array([np.inf, -np.inf], np.float32), fmt)
        nan = np.array([0x7E00 if fmt == "f16" else 0x7FC0], np.uint16)
        h = np.concatenate([h, specials, nan])
        xv = _widen_lib(h, fmt).astype(np.float64)
        f = None if fmt == "f16" else "bf16"
        any_, mn, mx = O.value_range(_as_input(h, fmt), fmt=f)
        assert any_ and mn == np.nanmin(xv[:3]) and mx == np.nanmax(xv[:3])
        c = O.consts("noa", fmt, 1e-3, x=_as_input(h, fmt))
        assert c.R == mx - mn  # exact: both are 16-bit values
    h = np.array([0x7C00, 0xFC00, 0x7E00] if fmt == "f16" else [0x7F80, 0xFF80, 0x7FC0], np.uint16)
    c = O.consts("noa", fmt, 1e-3, x=_as_input(h, fmt))
    assert c.all_outliers == 1


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_signed_zero_and_tiny_abs_values(fmt):
    h = np.array([0x0000, 0x8000, 0x0001, 0x8001], np.uint16)
    f = None if fmt == "f16" else "bf16"
    q = O.quantize(_as_input(h, fmt), "abs", 1e-3, fmt=f)
    assert q.count == 0 and np.all(q.bins == 0)
    assert np.all(O.dequantize(q).view(np.uint16) == 0)  # +0 (reading R7)


def test_dtype_errors():
    with pytest.raises(TypeError):
        O.quantize(np.zeros(4, np.uint16), "abs", 1e-3)
    with pytest.raises(TypeError):
        O.quantize(np.zeros(4, np.float32), "abs", 1e-3, fmt="bf16")
    with pytest.raises(TypeError):
        O.quantize_unprotected(np.zeros(4, np.float16), 1e-3)
