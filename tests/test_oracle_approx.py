"""Pins of the oracle's log2/pow2 approximations (Sec. 3.2) to their closed forms.

For a positive normal float a = 2^(E-127) (1 + M 2^-23) the approximation is the
piecewise-linear log2approx(a) = RN_f32(E - 127 + M 2^-23); its inverse maps L to
2^(k-127) (1 + bb - k) with bb = RN_f32(L + 127), k = floor(bb).  Both closed
forms are evaluated here with exact float64 / rational arithmetic, which is
independent of the bit manipulations the oracle uses.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O


def _normals_f32(exps, mant_stride, rng=None):
    M = np.arange(0, 1 << 23, mant_stride, dtype=np.uint32)
    if rng is not None:
        M = np.unique(np.concatenate([M, rng.integers(0, 1 << 23, 4096).astype(np.uint32),
                                      np.array([0, 1, (1 << 22), (1 << 23) - 1], np.uint32)]))
    E = np.asarray(exps, dtype=np.uint32)
    bits = (E[:, None] << 23) | M[None, :]
    return bits.reshape(-1).view(np.float32), (E[:, None] + 0 * M[None, :]).reshape(-1), \
        np.broadcast_to(M[None, :], (len(E), len(M))).reshape(-1)


def _log2_closed_f32(E, M):
    exact = (E.astype(np.float64) - 127.0) + M.astype(np.float64) * 2.0 ** -23  # exact in f64
    return exact.astype(np.float32)  # one round-to-nearest


def test_log2approx_f32_powers_of_two():
    for k in range(-126, 128):
        assert O.log2approx_f32(math.ldexp(1.0, k)) == k


def test_log2approx_f32_closed_form_all_exponents():
    rng = np.random.default_rng(1)
    a, E, M = _normals_f32(range(1, 255), 1 << 10, rng)
    got = O.log2approx_f32_array(a)
    assert np.array_equal(got.view(np.uint32), _log2_closed_f32(E, M).view(np.uint32))


def test_log2approx_f32_closed_form_dense_exponents():
    # every mantissa for the smallest, unit and largest binades
    a, E, M = _normals_f32([1, 100, 127, 128, 254], 1)
    got = O.log2approx_f32_array(a)
    assert np.array_equal(got.view(np.uint32), _log2_closed_f32(E, M).view(np.uint32))


def test_log2approx_f32_monotone():
    rng = np.random.default_rng(2)
    a, _, _ = _normals_f32(range(1, 255), 1 << 12, rng)
    a = np.sort(a)
    L = O.log2approx_f32_array(a)
    assert np.all(np.diff(L.astype(np.float64)) >= 0)


def _pow2_closed_f32(L):
    bb = (L.astype(np.float32) + np.float32(127.0)).astype(np.float64)  # RN_f32(L + 127)
    k = np.floor(bb)
    return np.ldexp(1.0 + (bb - k), (k - 127).astype(np.int64)).astype(np.float32), bb


def test_pow2approx_f32_integers():
    for k in range(-126, 128):
        assert O.pow2approx_f32(float(k)) == math.ldexp(1.0, k)


def test_pow2approx_f32_closed_form():
    rng = np.random.default_rng(3)
    L = np.concatenate([
        rng.uniform(-126.0, 127.999, 1 << 20),
        np.arange(-126, 128, dtype=np.float64) + 0.5,
        np.array([-126.0, 127.99998, 0.0, -0.0, 1e-7, -1e-7]),
    ]).astype(np.float32)
    want, bb = _pow2_closed_f32(L)
    keep = (bb >= 1.0) & (bb < 255.0)
    got = O.pow2approx_f32_array(L[keep])
    assert np.array_equal(got.view(np.uint32), want[keep].view(np.uint32))


def test_pow2approx_inverts_log2approx_where_exact():
    # Where L = log2approx(a) and L + 127 are exact, pow2approx returns a.
    rng = np.random.default_rng(4)
    for e in range(-20, 21):
        M = rng.integers(0, 1 << 10, 64).astype(np.uint32) << 13  # 10 mantissa bits
        a = ((np.uint32(e + 127) << 23) | M).view(np.float32)
        L = O.log2approx_f32_array(a)
        back = O.pow2approx_f32_array(L)
        assert np.array_equal(back.view(np.uint32), a.view(np.uint32))


def test_log2approx_f64_closed_form():
    rng = np.random.default_rng(5)
    for _ in range(4000):
        E = int(rng.integers(1, 2047))
        M = int(rng.integers(0, 1 << 52))
        a = np.array([(E << 52) | M], dtype=np.uint64).view(np.float64)[0]
        want = float(Fraction(E - 1023) + Fraction(M, 1 << 52))  # correctly rounded
        assert O.log2approx_f64(a) == want
    for k in (-1022, -1, 0, 1, 52, 1023):
        assert O.log2approx_f64(math.ldexp(1.0, k)) == k


def test_pow2approx_f64_closed_form():
    rng = np.random.default_rng(6)
    Ls = list(rng.uniform(-1022.0, 1023.999, 4000)) + [float(k) for k in range(-1022, 1024, 97)]
    for L in Ls:
        bb = L + 1023.0
        if not (1.0 <= bb < 2047.0):
            continue
        k = math.floor(bb)
        want = math.ldexp(1.0 + (bb - k), k - 1023)
        assert O.pow2approx_f64(L) == want
    for k in range(-1022, 1024, 31):
        assert O.pow2approx_f64(float(k)) == math.ldexp(1.0, k)


@pytest.mark.slow
def test_log2approx_f32_closed_form_exhaustive():
    for E in range(1, 255):
        a, Ee, M = _normals_f32([E], 1)
        got = O.log2approx_f32_array(a)
        assert np.array_equal(got.view(np.uint32), _log2_closed_f32(Ee, M).view(np.uint32)), E
