"""CPU oracle for the guaranteed-error-bound quantizers (arXiv 2407.15037).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg use this package; the product path (the CUDA library and its
binding) never imports it.  The numerical work is the plain scalar C code in
lcq_oracle.c; this module only marshals numpy arrays.

Parity is unpinned for nothing in this module: every function is checked in
tests/test_oracle_*.py against closed forms, exact rational arithmetic, brute
force or the bound definitions of Sec. 2.1.
"""
import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

F32, F64, F16, BF16 = 0, 1, 2, 3
ABS, REL, NOA = 0, 1, 2
BOUND_NAMES = {"abs": ABS, "rel": REL, "noa": NOA}
DTYPES = {np.dtype(np.float32): F32, np.dtype(np.float64): F64, np.dtype(np.float16): F16}
# numpy has no bfloat16: bfloat16 arrays travel as uint16 bit patterns with
# fmt="bf16" (binary16 arrays may be float16, or uint16 with fmt="f16")
FORMATS = {"f16": F16, "bf16": BF16}
PAYLOAD = {F32: np.uint32, F64: np.uint64, F16: np.uint16, BF16: np.uint16}


class Consts(ctypes.Structure):
    _fields_ = [
        ("dtype", ctypes.c_int32), ("bound", ctypes.c_int32),
        ("all_outliers", ctypes.c_int32), ("pad", ctypes.c_int32),
        ("eb", ctypes.c_double), ("R", ctypes.c_double), ("eb_abs", ctypes.c_double),
        ("ebT", ctypes.c_double), ("eb2", ctypes.c_double), ("inv", ctypes.c_double),
        ("lb", ctypes.c_double), ("step", ctypes.c_double), ("inv_l", ctypes.c_double),
        ("chk", ctypes.c_double),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "pad"}


_lib = None
_lock = threading.Lock()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            vp, u64, i32, dbl = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double
            P = ctypes.POINTER
            L.lcqo_fp_env_ok.restype = ctypes.c_int
            L.lcqo_log2approx_f32.argtypes = [ctypes.c_float]
            L.lcqo_log2approx_f32.restype = ctypes.c_float
            L.lcqo_pow2approx_f32.argtypes = [ctypes.c_float]
            L.lcqo_pow2approx_f32.restype = ctypes.c_float
            L.lcqo_log2approx_f64.argtypes = [dbl]
            L.lcqo_log2approx_f64.restype = dbl
            L.lcqo_pow2approx_f64.argtypes = [dbl]
            L.lcqo_pow2approx_f64.restype = dbl
            for fn in (L.lcqo_consts_abs, L.lcqo_consts_rel):
                fn.argtypes = [ctypes.c_int, dbl, P(Consts)]
                fn.restype = ctypes.c_int
            L.lcqo_consts_noa.argtypes = [ctypes.c_int, dbl, vp, u64, P(Consts)]
            L.lcqo_consts_noa.restype = ctypes.c_int
            L.lcqo_consts_noa_from_range.argtypes = [ctypes.c_int, dbl, i32, dbl, dbl, P(Consts)]
            L.lcqo_consts_noa_from_range.restype = ctypes.c_int
            L.lcqo_range.argtypes = [ctypes.c_int, vp, u64, P(i32), P(dbl), P(dbl)]
            L.lcqo_range.restype = None
            L.lcqo_quantize.argtypes = [P(Consts), vp, u64, vp, vp, vp, u64]
            L.lcqo_quantize.restype = u64
            L.lcqo_dequantize.argtypes = [P(Consts), vp, vp, vp, u64, vp]
            L.lcqo_dequantize.restype = None
            L.lcqo_quantize_unprotected.argtypes = [P(Consts), vp, u64, vp, vp, vp, u64]
            L.lcqo_quantize_unprotected.restype = u64
            L.lcqo_rel_library_recon.argtypes = [ctypes.c_int, dbl, vp, vp, u64, vp]
            L.lcqo_rel_library_recon.restype = None
            L.lcqo_verify_abs.argtypes = [ctypes.c_int, vp, vp, u64, dbl]
            L.lcqo_verify_abs.restype = u64
            L.lcqo_verify_rel.argtypes = [ctypes.c_int, vp, vp, u64, dbl]
            L.lcqo_verify_rel.restype = u64
            for nm in ("lcqo_log2approx_f32_array", "lcqo_pow2approx_f32_array",
                       "lcqo_log2approx_f64_array", "lcqo_pow2approx_f64_array"):
                getattr(L, nm).argtypes = [vp, vp, u64]
                getattr(L, nm).restype = None
            L.lcqo_sweep_f32.argtypes = [P(Consts), u64, u64, dbl, P(u64)]
            L.lcqo_sweep_f32.restype = None
            L.lcqo_widen16_array.argtypes = [ctypes.c_int, vp, vp, u64]
            L.lcqo_widen16_array.restype = None
            L.lcqo_round16_array.argtypes = [ctypes.c_int, vp, vp, u64]
            L.lcqo_round16_array.restype = None
            _lib = L
    if not _lib.lcqo_fp_env_ok():
        raise RuntimeError("oracle: FTZ/DAZ set or rounding mode is not to-nearest")
    return _lib


class BoundError(ValueError):
    pass


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if a is not None and a.size else ctypes.c_void_p(0)


def _dtype_code(x, fmt=None):
    if fmt is not None:
        if FORMATS[fmt] == F16 and np.dtype(x.dtype) == np.float16:
            return F16
        if np.dtype(x.dtype) != np.uint16:
            raise TypeError("oracle: fmt=%r takes uint16 bit patterns" % fmt)
        return FORMATS[fmt]
    try:
        return DTYPES[np.dtype(x.dtype)]
    except KeyError:
        raise TypeError("oracle: float32, float64 or float16 input required (bfloat16: uint16 bits, "
                        "fmt='bf16')") from None


def _fmt_of(code):
    return {F16: "f16", BF16: "bf16"}.get(code)


def dtype_code(dtype):
    """Oracle dtype code of a numpy float dtype or of 'f16' / 'bf16'."""
    if isinstance(dtype, str) and dtype in FORMATS:
        return FORMATS[dtype]
    return DTYPES[np.dtype(dtype)]


def consts(bound, dtype, eb, x=None, rng=None):
    """Derived constants (Sec. 2.2 and readings R2-R6, R11).

    bound: 'abs' | 'rel' | 'noa'; dtype: numpy float dtype, or 'f16' /
    'bf16'; for NOA give the input x, or rng=(any_finite, mn, mx) for a range
    computed elsewhere.
    """
    b = BOUND_NAMES[bound] if isinstance(bound, str) else bound
    d = dtype_code(dtype)
    c = Consts()
    L = lib()
    if b == ABS:
        st = L.lcqo_consts_abs(d, float(eb), ctypes.byref(c))
    elif b == REL:
        st = L.lcqo_consts_rel(d, float(eb), ctypes.byref(c))
    elif rng is not None:
        st = L.lcqo_consts_noa_from_range(d, float(eb), int(rng[0]), float(rng[1]), float(rng[2]),
                                          ctypes.byref(c))
    else:
        x = np.ascontiguousarray(x)
        if _dtype_code(x, _fmt_of(d)) != d:
            raise TypeError("oracle: input does not match dtype %r" % (dtype,))
        st = L.lcqo_consts_noa(d, float(eb), _ptr(x), x.size, ctypes.byref(c))
    if st != 0:
        raise BoundError("oracle: bound %r rejected (status %d)" % (eb, st))
    return c


def value_range(x, fmt=None):
    """(any_finite, min, max) over the finite values of x (reading R6)."""
    x = np.ascontiguousarray(x)
    any_ = ctypes.c_int32()
    mn, mx = ctypes.c_double(), ctypes.c_double()
    lib().lcqo_range(_dtype_code(x, fmt), _ptr(x), x.size, ctypes.byref(any_), ctypes.byref(mn),
                     ctypes.byref(mx))
    return bool(any_.value), mn.value, mx.value


@dataclass
class Quantized:
    bins: np.ndarray      # int32[n]
    mask: np.ndarray      # uint32[ceil(n/32)]
    payload: np.ndarray   # uint32, uint64 or uint16 [count] (raw bits)
    count: int
    consts: Consts


def quantize_with(c, x, capacity=None):
    """Quantize x with precomputed constants c (bins, mask, payload, count)."""
    x = np.ascontiguousarray(x)
    if _dtype_code(x, _fmt_of(c.dtype)) != c.dtype:
        raise TypeError("oracle: dtype does not match the constants")
    n = x.size
    cap = n if capacity is None else int(capacity)
    bins = np.empty(n, dtype=np.int32)
    mask = np.empty((n + 31) // 32, dtype=np.uint32)
    pay = np.empty(max(cap, 0), dtype=PAYLOAD[c.dtype])
    cnt = lib().lcqo_quantize(ctypes.byref(c), _ptr(x), n, _ptr(bins), _ptr(mask), _ptr(pay), cap)
    return Quantized(bins, mask, pay[:min(cnt, cap)], int(cnt), c)


def quantize(x, bound, eb, capacity=None, fmt=None):
    """fmt: None (x is float32/64/16), or 'f16' / 'bf16' for uint16 bits."""
    x = np.ascontiguousarray(x)
    d = _dtype_code(x, fmt)
    c = consts(bound, _fmt_of(d) or x.dtype, eb, x=x)
    return quantize_with(c, x, capacity)


def dequantize(q):
    """Decoded values: float32 / float64 / float16 arrays; bfloat16 as uint16
    bit patterns."""
    c = q.consts
    n = q.bins.size
    out = np.empty(n, dtype={F32: np.float32, F64: np.float64, F16: np.float16, BF16: np.uint16}[c.dtype])
    lib().lcqo_dequantize(ctypes.byref(c), _ptr(q.bins), _ptr(q.mask), _ptr(q.payload), n,
                          _ptr(out))
    return out


def quantize_unprotected(x, eb):
    """Ablation: ABS without the reconstruct-and-check step (Sec. 6, Tables
    7-8); the result decodes with dequantize() like any ABS result."""
    x = np.ascontiguousarray(x)
    if _dtype_code(x) not in (F32, F64):
        raise TypeError("oracle: the ablations take float32 or float64")
    c = consts("abs", x.dtype, eb)
    n = x.size
    bins = np.empty(n, dtype=np.int32)
    mask = np.empty((n + 31) // 32, dtype=np.uint32)
    pay = np.empty(n, dtype=np.uint32 if c.dtype == F32 else np.uint64)
    cnt = lib().lcqo_quantize_unprotected(ctypes.byref(c), _ptr(x), n, _ptr(bins), _ptr(mask), _ptr(pay), n)
    return Quantized(bins, mask, pay[:cnt], int(cnt), c)


def rel_library_recon(dtype, step, bins, mask):
    """Ablation: decode REL bins with the host C library's exp2 (Sec. 2.3);
    0 where the mask marks an outlier."""
    bins = np.ascontiguousarray(bins, dtype=np.int32)
    mask = np.ascontiguousarray(mask, dtype=np.uint32)
    dt = np.dtype(dtype)
    out = np.empty(bins.size, dtype=dt)
    lib().lcqo_rel_library_recon(DTYPES[dt], float(step), _ptr(bins), _ptr(mask), bins.size, _ptr(out))
    return out


def verify_abs(x, xr, eb, fmt=None):
    """Exact count of elements with |x - x'| > eb (Sec. 2.1.1); 0 means sound."""
    x, xr = np.ascontiguousarray(x), np.ascontiguousarray(xr)
    d = _dtype_code(x, fmt)
    if _dtype_code(xr, fmt) != d or xr.size != x.size:
        raise TypeError("oracle: x and x' differ in type or size")
    return int(lib().lcqo_verify_abs(d, _ptr(x), _ptr(xr), x.size, float(eb)))


def verify_rel(x, xr, eps, fmt=None):
    """Exact count of elements outside |x|/(1+eps) <= |x'| <= |x|(1+eps) with
    equal sign (Sec. 2.1.2); bit-identical reconstructions always pass."""
    x, xr = np.ascontiguousarray(x), np.ascontiguousarray(xr)
    d = _dtype_code(x, fmt)
    if _dtype_code(xr, fmt) != d or xr.size != x.size:
        raise TypeError("oracle: x and x' differ in type or size")
    return int(lib().lcqo_verify_rel(d, _ptr(x), _ptr(xr), x.size, float(eps)))


def widen16(h, fmt):
    """The float32 values of 16-bit patterns h (uint16) in format fmt (R11)."""
    h = np.ascontiguousarray(h, dtype=np.uint16)
    out = np.empty(h.size, dtype=np.float32)
    lib().lcqo_widen16_array(FORMATS[fmt], _ptr(h), _ptr(out), h.size)
    return out


def round16(x, fmt):
    """float32 values (not NaN) rounded to nearest-even in format fmt; uint16
    bit patterns (R11)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(x.size, dtype=np.uint16)
    lib().lcqo_round16_array(FORMATS[fmt], _ptr(x), _ptr(out), x.size)
    return out


def _verify_parallel(fn, x, xr, eb, threads=None):
    x, xr = np.ascontiguousarray(x), np.ascontiguousarray(xr)
    threads = threads or os.cpu_count() or 1
    step = max(1, (x.size + threads - 1) // threads)
    res = [0] * threads

    def run(k):
        s = k * step
        e = min(x.size, s + step)
        res[k] = fn(x[s:e], xr[s:e], eb) if e > s else 0

    ts = [threading.Thread(target=run, args=(k,)) for k in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return sum(res)


def verify_abs_parallel(x, xr, eb, threads=None):
    """verify_abs over contiguous slices on host threads (same count)."""
    return _verify_parallel(verify_abs, x, xr, eb, threads)


def verify_rel_parallel(x, xr, eps, threads=None):
    """verify_rel over contiguous slices on host threads (same count)."""
    return _verify_parallel(verify_rel, x, xr, eps, threads)


def log2approx_f32(a):
    return lib().lcqo_log2approx_f32(float(a))


def pow2approx_f32(L):
    return lib().lcqo_pow2approx_f32(float(L))


def log2approx_f64(a):
    return lib().lcqo_log2approx_f64(float(a))


def pow2approx_f64(L):
    return lib().lcqo_pow2approx_f64(float(L))


def _array_fn(name, a, dt):
    a = np.ascontiguousarray(a, dtype=dt)
    out = np.empty_like(a)
    getattr(lib(), name)(_ptr(a), _ptr(out), a.size)
    return out


def log2approx_f32_array(a):
    return _array_fn("lcqo_log2approx_f32_array", a, np.float32)


def pow2approx_f32_array(L):
    return _array_fn("lcqo_pow2approx_f32_array", L, np.float32)


def log2approx_f64_array(a):
    return _array_fn("lcqo_log2approx_f64_array", a, np.float64)


def pow2approx_f64_array(L):
    return _array_fn("lcqo_pow2approx_f64_array", L, np.float64)


def sweep_f32(c, start, count, eb_verify):
    """Quantize, reconstruct and exactly verify float32 bit patterns
    [start, start+count).  Returns (outliers, violations, inexact)."""
    out = (ctypes.c_uint64 * 3)()
    lib().lcqo_sweep_f32(ctypes.byref(c), int(start), int(count), float(eb_verify), out)
    return tuple(int(v) for v in out)


def sweep_f32_parallel(c, start, count, eb_verify, threads=None):
    """sweep_f32 split across host threads (ctypes releases the GIL); the
    per-element results do not depend on the split."""
    threads = threads or os.cpu_count() or 1
    step = (count + threads - 1) // threads
    res = [None] * threads

    def run(k):
        s = start + k * step
        e = min(start + count, s + step)
        res[k] = sweep_f32(c, s, max(e - s, 0), eb_verify) if e > s else (0, 0, 0)

    ts = [threading.Thread(target=run, args=(k,)) for k in range(threads)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    return tuple(sum(r[i] for r in res) for i in range(3))


def quantize_parallel(c, x, threads=None, chunk_words=None):
    """quantize_with() over contiguous chunks on host threads, concatenated in
    index order (chunk boundaries are multiples of 32 elements so the mask
    words line up).  Used to keep large parity checks within seconds."""
    x = np.ascontiguousarray(x)
    n = x.size
    threads = threads or os.cpu_count() or 1
    per = max(32, ((n + threads - 1) // threads + 31) // 32 * 32)
    bounds = [(s, min(n, s + per)) for s in range(0, n, per)]
    parts = [None] * len(bounds)

    def run(k):
        s, e = bounds[k]
        parts[k] = quantize_with(c, x[s:e])

    ts = [threading.Thread(target=run, args=(k,)) for k in range(len(bounds))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    if not parts:
        return quantize_with(c, x)
    bins = np.concatenate([p.bins for p in parts])
    mask = np.concatenate([p.mask for p in parts])
    pay = np.concatenate([p.payload for p in parts])
    return Quantized(bins, mask, pay, int(sum(p.count for p in parts)), c)
