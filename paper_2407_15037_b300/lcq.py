"""Python binding of liblcq.so (include/lcq.h): argument marshalling only.

Every step of quantize / verify / compact / dequantize runs in the library's
CUDA kernels; PyTorch only provides device memory and streams.  There is no
CPU fallback: if the library cannot be loaded, or no CUDA device is present,
the calls raise.
"""
import ctypes
import os
from dataclasses import dataclass

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblcq.so")

F32, F64, F16, BF16 = 0, 1, 2, 3
DTYPE_CODES = {torch.float32: F32, torch.float64: F64, torch.float16: F16, torch.bfloat16: BF16}
# raw-bit tensor type of the outlier payload per data type
PAYLOAD_DTYPES = {torch.float32: torch.int32, torch.float64: torch.int64, torch.float16: torch.int16,
                  torch.bfloat16: torch.int16}
ABS, REL, NOA = 0, 1, 2
BOUNDS = {"abs": ABS, "rel": REL, "noa": NOA}
STATUS_CAPACITY, STATUS_TIMEOUT, STATUS_HEADER = 1, 2, 4
MAGIC = 0x3151434C

STATUS_NAMES = {0: "LCQ_OK", 1: "LCQ_ERR_ARG", 2: "LCQ_ERR_BOUND", 3: "LCQ_ERR_CAPACITY",
                4: "LCQ_ERR_TIMEOUT", 5: "LCQ_ERR_CUDA", 6: "LCQ_ERR_WORKSPACE",
                7: "LCQ_ERR_HEADER"}


class Header(ctypes.Structure):
    """Mirror of struct lcq_header."""
    _fields_ = [
        ("magic", ctypes.c_uint32), ("dtype", ctypes.c_uint32), ("bound_type", ctypes.c_uint32),
        ("mode", ctypes.c_uint32), ("n", ctypes.c_uint64), ("eb", ctypes.c_double),
        ("range", ctypes.c_double), ("eb_abs", ctypes.c_double), ("ebT_bits", ctypes.c_uint64),
        ("scale_bits", ctypes.c_uint64), ("inv_bits", ctypes.c_uint64), ("chk_bits", ctypes.c_uint64),
        ("outlier_count", ctypes.c_uint64), ("status", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
    ]


HEADER_BYTES = ctypes.sizeof(Header)


class BatchItem(ctypes.Structure):
    """Mirror of struct lcq_batch_item."""
    _fields_ = [
        ("dtype", ctypes.c_uint32), ("bound_type", ctypes.c_uint32), ("eb", ctypes.c_double),
        ("n", ctypes.c_uint64), ("d_in", ctypes.c_void_p), ("d_bins", ctypes.c_void_p),
        ("d_mask", ctypes.c_void_p), ("d_outliers", ctypes.c_void_p),
        ("outlier_capacity", ctypes.c_uint64), ("d_hdr", ctypes.c_void_p),
    ]


class BatchInfo(ctypes.Structure):
    """Mirror of struct lcq_batch_info."""
    _fields_ = [
        ("count", ctypes.c_uint32), ("noa_count", ctypes.c_uint32), ("total_tiles", ctypes.c_uint64),
        ("noa_chunks", ctypes.c_uint64), ("total_values", ctypes.c_uint64),
        ("total_bytes_in", ctypes.c_uint64), ("bad_item", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
    ]


class HostItem(ctypes.Structure):
    """Mirror of struct lcq_host_item."""
    _fields_ = [("dtype", ctypes.c_uint32), ("bound_type", ctypes.c_uint32), ("eb", ctypes.c_double),
                ("h_in", ctypes.c_void_p), ("n", ctypes.c_uint64), ("h_bins", ctypes.c_void_p),
                ("h_mask", ctypes.c_void_p), ("h_outliers", ctypes.c_void_p),
                ("outlier_capacity", ctypes.c_uint64), ("h_hdr", ctypes.c_void_p),
                ("status", ctypes.c_int32), ("reserved", ctypes.c_uint32)]


class LcqError(RuntimeError):
    def __init__(self, code, what):
        super().__init__("%s failed: %s" % (what, STATUS_NAMES.get(code, str(code))))
        self.code = code


# Exported symbols and their ctypes signatures (must match include/lcq.h).
_vp, _u64, _u32, _i32, _dbl, _sz = (ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                                     ctypes.c_int32, ctypes.c_double, ctypes.c_size_t)
SIGNATURES = {
    "lcq_workspace_size": ([ctypes.c_int, ctypes.c_int, _u64], _sz),
    "lcq_workspace_init": ([_vp, _sz, _vp], ctypes.c_int),
    "lcq_quantize": ([ctypes.c_int, ctypes.c_int, _dbl, _vp, _u64, _vp, _vp, _vp, _u64, _vp, _vp,
                      _sz, _vp], ctypes.c_int),
    "lcq_dequantize": ([ctypes.c_int, _u64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp],
                       ctypes.c_int),
    "lcq_finite_range": ([ctypes.c_int, _vp, _u64, _vp, _vp, _sz, _vp], ctypes.c_int),
    "lcq_quantize_noa_range": ([ctypes.c_int, _dbl, ctypes.c_int, _dbl, _dbl, _vp, _u64, _vp, _vp, _vp, _u64,
                                _vp, _vp, _sz, _vp], ctypes.c_int),
    "lcq_quantize_ablation": ([ctypes.c_int, ctypes.c_int, _dbl, _vp, _u64, _vp, _vp, _vp, _u64, _vp, _vp, _sz,
                               _vp], ctypes.c_int),
    "lcq_ablation_variant": ([ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "lcq_rel_library_reconstruct": ([ctypes.c_int, _u64, _vp, _vp, _vp, _vp, _vp, _vp], ctypes.c_int),
    "lcq_count_abs_violations": ([ctypes.c_int, _dbl, _vp, _vp, _u64, _vp, _vp], ctypes.c_int),
    "lcq_sync_status": ([_vp, _vp, _vp], ctypes.c_int),
    "lcq_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "lcq_host_stage_size": ([ctypes.c_int, _u64, _u64], _sz),
    "lcq_quantize_host": ([ctypes.c_int, ctypes.c_int, _dbl, _vp, _u64, _vp, _vp, _vp, _u64, _vp,
                           _vp, _sz, _vp, _sz, _vp], ctypes.c_int),
    "lcq_host_batch_stage_size": ([_vp, _u32], _sz),
    "lcq_quantize_host_batch": ([_vp, _u32, _vp, _sz, _vp, _sz, _vp], ctypes.c_int),
    "lcq_pack_bound": ([_u64], _sz),
    "lcq_pack_workspace_size": ([_u64], _sz),
    "lcq_pack": ([_vp, _u64, _vp, _sz, _vp, _vp, _sz, _vp], ctypes.c_int),
    "lcq_unpack": ([_vp, _sz, _u64, _vp, _vp, _vp, _sz, _vp], ctypes.c_int),
    "lcq_debug_set_scan": ([_u32, _u64], None),
    "lcq_tune_variant_count": ([], ctypes.c_int),
    "lcq_tune_describe": ([ctypes.c_int, _vp, _vp, _vp, _vp], ctypes.c_int),
    "lcq_tune_set": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "lcq_tune_get": ([ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "lcq_autotune_quantize": ([ctypes.c_int, ctypes.c_int, _dbl, _vp, _u64, _vp, _vp, _vp, _u64, _vp,
                               _vp, _sz, _vp, ctypes.c_int, _vp], ctypes.c_int),
    "lcq_autotune_dequantize": ([ctypes.c_int, _u64, _vp, _vp, _vp, _vp, _vp, _vp, _sz, _vp,
                                 ctypes.c_int, _vp], ctypes.c_int),
    "lcq_batch_plan_size": ([_u32], _sz),
    "lcq_batch_workspace_size": ([_vp, _u32], _sz),
    "lcq_batch_prepare": ([_vp, _u32, _vp, _sz, _vp, _sz, _vp, _vp], ctypes.c_int),
    "lcq_quantize_batched": ([_vp, _vp, _vp, _sz, _vp], ctypes.c_int),
    "lcq_batch_tune_variant_count": ([], ctypes.c_int),
    "lcq_batch_tune_set": ([ctypes.c_int], ctypes.c_int),
    "lcq_batch_tune_get": ([], ctypes.c_int),
    "lcq_autotune_batched": ([_vp, _vp, _vp, _sz, _vp, ctypes.c_int, _vp], ctypes.c_int),
    "lcq_probe_fp64_mul": ([ctypes.c_uint32, ctypes.c_uint32, _vp, ctypes.POINTER(_u64), _vp], ctypes.c_int),
    "lcq_noalloc_max_values": ([], _u64),
    "lcq_quantize_noalloc": ([ctypes.c_int, ctypes.c_int, _dbl, _vp, _u64, _vp, _vp, _vp, _u64, _vp,
                              _vp], ctypes.c_int),
}

_lib = None


def lib():
    """Load liblcq.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("liblcq.so not built: run python -m paper_2407_15037_b300.build "
                              "(or __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(code, what):
    if code != 0:
        raise LcqError(code, what)


def _dtype_code(t):
    try:
        return DTYPE_CODES[t.dtype]
    except KeyError:
        raise TypeError("lcq: float32, float64, float16 or bfloat16 tensor required, got %s"
                        % t.dtype) from None


def _bound_code(bound):
    return BOUNDS[bound] if isinstance(bound, str) else int(bound)


def _stream_ptr(stream, device):
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() else ctypes.c_void_p(0)


def _require_cuda(t):
    if not t.is_cuda:
        raise ValueError("lcq: device tensors required (use quantize_host for host data)")


def workspace_size(dtype_code, bound, n):
    return int(lib().lcq_workspace_size(dtype_code, _bound_code(bound), int(n)))


def new_workspace(n, device, dtype_code=F32, bound=None):
    """A zero-filled workspace for arrays of up to n values (bound None:
    large enough for every bound type of this data type, so that float32
    REL stages its outliers)."""
    bounds = (ABS, REL, NOA) if bound is None else (bound,)
    nbytes = max(max(workspace_size(dtype_code, b, n) for b in bounds), 256)
    return torch.zeros(nbytes, dtype=torch.uint8, device=device)


@dataclass
class Quantized:
    """Device-resident compressed form (see include/lcq.h)."""
    bins: torch.Tensor      # int32[n]
    mask: torch.Tensor      # int32[ceil(n/32)] (raw uint32 words)
    outliers: torch.Tensor  # int32 / int64 / int16 [capacity] raw bit patterns
    header: torch.Tensor    # uint8[HEADER_BYTES] (struct lcq_header)
    n: int
    dtype: torch.dtype

    def read_header(self, stream=None):
        """Copy the header to the host (synchronises the stream)."""
        h = Header()
        raw = self.header.cpu() if stream is None else self.header.to("cpu", non_blocking=False)
        ctypes.memmove(ctypes.addressof(h), raw.numpy().ctypes.data, HEADER_BYTES)
        return h


def alloc_outputs(n, dtype, device, outlier_capacity=None):
    cap = n if outlier_capacity is None else int(outlier_capacity)
    if dtype not in PAYLOAD_DTYPES:
        raise TypeError("lcq: float32, float64, float16 or bfloat16 required, got %s" % dtype)
    pay_dtype = PAYLOAD_DTYPES[dtype]
    return Quantized(
        bins=torch.empty(n, dtype=torch.int32, device=device),
        mask=torch.empty((n + 31) // 32, dtype=torch.int32, device=device),
        outliers=torch.empty(cap, dtype=pay_dtype, device=device),
        header=torch.empty(HEADER_BYTES, dtype=torch.uint8, device=device),
        n=n, dtype=dtype)


def quantize_into(x, bound, eb, q, ws, stream=None):
    """Enqueue lcq_quantize of the contiguous device tensor x into the
    preallocated outputs q, using workspace ws.  No host synchronisation."""
    _require_cuda(x)
    code = lib().lcq_quantize(
        _dtype_code(x), _bound_code(bound), float(eb), _ptr(x), x.numel(), _ptr(q.bins),
        _ptr(q.mask), _ptr(q.outliers), q.outliers.numel(), _ptr(q.header), _ptr(ws), ws.numel(),
        _stream_ptr(stream, x.device))
    _check(code, "lcq_quantize")
    return q


def quantize(x, bound, eb, outlier_capacity=None, ws=None, stream=None):
    """Quantize a contiguous float32 / float64 / float16 / bfloat16 CUDA tensor
    with bound type 'abs' | 'rel' | 'noa' and bound eb.  Returns the
    device-resident result."""
    _require_cuda(x)
    x = x.contiguous().reshape(-1)
    q = alloc_outputs(x.numel(), x.dtype, x.device, outlier_capacity)
    if ws is None:
        ws = new_workspace(x.numel(), x.device, _dtype_code(x), bound)
    return quantize_into(x, bound, eb, q, ws, stream)


def quantize_noalloc_into(x, bound, eb, q, stream=None):
    """Enqueue lcq_quantize_noalloc (no workspace argument; the library's
    built-in scratch of x's device is used, so the call runs with that device
    current).  Calls on one device must not overlap."""
    _require_cuda(x)
    with torch.cuda.device(x.device):
        code = lib().lcq_quantize_noalloc(
            _dtype_code(x), _bound_code(bound), float(eb), _ptr(x), x.numel(), _ptr(q.bins),
            _ptr(q.mask), _ptr(q.outliers), q.outliers.numel(), _ptr(q.header),
            _stream_ptr(stream, x.device))
    _check(code, "lcq_quantize_noalloc")
    return q


def finite_range(x, ws=None, stream=None):
    """Enqueue lcq_finite_range; returns a float64 device tensor
    {has_finite, min, max} (no host synchronisation)."""
    _require_cuda(x)
    x = x.reshape(-1)
    if ws is None:
        ws = new_workspace(x.numel(), x.device, _dtype_code(x), NOA)
    out = torch.empty(3, dtype=torch.float64, device=x.device)
    code = lib().lcq_finite_range(_dtype_code(x), _ptr(x), x.numel(), _ptr(out), _ptr(ws), ws.numel(),
                                  _stream_ptr(stream, x.device))
    _check(code, "lcq_finite_range")
    return out


def quantize_noa_range_into(x, eb, rng, q, ws, stream=None):
    """Enqueue lcq_quantize_noa_range: NOA with the caller's finite range
    rng = (has_finite, min, max) (host values)."""
    _require_cuda(x)
    has, mn, mx = rng
    code = lib().lcq_quantize_noa_range(
        _dtype_code(x), float(eb), 1 if has else 0, float(mn) if has else 0.0, float(mx) if has else 0.0,
        _ptr(x), x.numel(), _ptr(q.bins), _ptr(q.mask), _ptr(q.outliers), q.outliers.numel(), _ptr(q.header),
        _ptr(ws), ws.numel(), _stream_ptr(stream, x.device))
    _check(code, "lcq_quantize_noa_range")
    return q


ABLATIONS = {"abs_no_check": 0, "rel_library": 1}


def quantize_ablation_into(x, kind, eb, q, ws, stream=None):
    """Enqueue lcq_quantize_ablation ('abs_no_check' | 'rel_library')."""
    _require_cuda(x)
    code = lib().lcq_quantize_ablation(
        ABLATIONS[kind], _dtype_code(x), float(eb), _ptr(x), x.numel(), _ptr(q.bins), _ptr(q.mask),
        _ptr(q.outliers), q.outliers.numel(), _ptr(q.header), _ptr(ws), ws.numel(), _stream_ptr(stream, x.device))
    _check(code, "lcq_quantize_ablation")
    return q


def quantize_ablation(x, kind, eb, ws=None, stream=None):
    _require_cuda(x)
    x = x.contiguous().reshape(-1)
    q = alloc_outputs(x.numel(), x.dtype, x.device)
    if ws is None:
        ws = new_workspace(x.numel(), x.device, _dtype_code(x))
    return quantize_ablation_into(x, kind, eb, q, ws, stream)


def ablation_variant(dtype_code, kind):
    return int(lib().lcq_ablation_variant(dtype_code, ABLATIONS[kind]))


def rel_library_reconstruct(q, out=None, stream=None, check=True):
    """Library-exp2 decode of a 'rel_library' result (0 at outliers)."""
    if out is None:
        out = torch.empty(q.n, dtype=q.dtype, device=q.bins.device)
    status = torch.zeros(1, dtype=torch.int32, device=out.device)
    code = lib().lcq_rel_library_reconstruct(_dtype_code(out), q.n, _ptr(q.header), _ptr(q.bins), _ptr(q.mask),
                                             _ptr(out), _ptr(status), _stream_ptr(stream, out.device))
    _check(code, "lcq_rel_library_reconstruct")
    if check and int(status.item()):
        raise LcqError(7, "lcq_rel_library_reconstruct (device status %d)" % int(status.item()))
    return out


def count_abs_violations(x, xr, eb, stream=None):
    """Number of i with |x_i - xr_i| > eb in exact arithmetic (synchronises)."""
    _require_cuda(x)
    cnt = torch.empty(1, dtype=torch.int64, device=x.device)
    code = lib().lcq_count_abs_violations(_dtype_code(x), float(eb), _ptr(x), _ptr(xr), x.numel(), _ptr(cnt),
                                          _stream_ptr(stream, x.device))
    _check(code, "lcq_count_abs_violations")
    return int(cnt.item())


def dequantize_into(q, out, ws, status=None, stream=None):
    _require_cuda(out)
    code = lib().lcq_dequantize(
        _dtype_code(out), q.n, _ptr(q.header), _ptr(q.bins), _ptr(q.mask), _ptr(q.outliers),
        _ptr(out), _ptr(status), _ptr(ws), ws.numel(), _stream_ptr(stream, out.device))
    _check(code, "lcq_dequantize")
    return out


def dequantize(q, ws=None, stream=None, check=True):
    """Reconstruct the values of a Quantized result on the device."""
    out = torch.empty(q.n, dtype=q.dtype, device=q.bins.device)
    if ws is None:
        ws = new_workspace(q.n, out.device)
    status = torch.zeros(1, dtype=torch.int32, device=out.device)
    dequantize_into(q, out, ws, status, stream)
    if check:
        st = int(status.item())
        if st:
            raise LcqError(7 if st & STATUS_HEADER else 4, "lcq_dequantize (device status %d)" % st)
    return out


def sync_status(q, stream=None):
    """Synchronise and return (status_code, outlier_count) for a result."""
    cnt = ctypes.c_uint64()
    code = lib().lcq_sync_status(_ptr(q.header), ctypes.byref(cnt), _stream_ptr(stream, q.bins.device))
    return code, cnt.value


def variant_count():
    return int(lib().lcq_tune_variant_count())


def describe_variant(v):
    a = [ctypes.c_int() for _ in range(4)]
    _check(lib().lcq_tune_describe(int(v), *[ctypes.byref(x) for x in a]), "lcq_tune_describe")
    return dict(vpt=a[0].value, stages=a[1].value, sub=a[2].value, min_ctas_per_sm=a[3].value)


def set_variant(kind, dtype_code, bound, v):
    _check(lib().lcq_tune_set(int(kind), int(dtype_code), _bound_code(bound), int(v)), "lcq_tune_set")


def get_variant(kind, dtype_code, bound):
    return int(lib().lcq_tune_get(int(kind), int(dtype_code), _bound_code(bound)))


def autotune_quantize(x, bound, eb, q, ws, reps=5, stream=None):
    """Time every tile-shape variant on this call and keep the fastest;
    returns the per-variant milliseconds."""
    nv = variant_count()
    ms = (ctypes.c_float * nv)()
    code = lib().lcq_autotune_quantize(
        _dtype_code(x), _bound_code(bound), float(eb), _ptr(x), x.numel(), _ptr(q.bins),
        _ptr(q.mask), _ptr(q.outliers), q.outliers.numel(), _ptr(q.header), _ptr(ws), ws.numel(),
        _stream_ptr(stream, x.device), int(reps), ms)
    _check(code, "lcq_autotune_quantize")
    return list(ms)


def autotune_dequantize(q, out, ws, reps=5, stream=None):
    nv = variant_count()
    ms = (ctypes.c_float * nv)()
    code = lib().lcq_autotune_dequantize(
        _dtype_code(out), q.n, _ptr(q.header), _ptr(q.bins), _ptr(q.mask), _ptr(q.outliers),
        _ptr(out), _ptr(ws), ws.numel(), _stream_ptr(stream, out.device), int(reps), ms)
    _check(code, "lcq_autotune_dequantize")
    return list(ms)


class Batch:
    """A prepared batch: the plan and workspace on the device plus the host
    info; keeps the input and output tensors alive.  `run()` enqueues
    lcq_quantize_batched (capturable in a CUDA graph)."""

    def __init__(self, arrays, device, stream=None):
        # arrays: list of (x, bound, eb, Quantized)
        self.arrays = arrays
        self.device = torch.device(device)
        n = len(arrays)
        items = (BatchItem * n)()
        for i, (x, bound, eb, q) in enumerate(arrays):
            _require_cuda(x)
            items[i] = BatchItem(_dtype_code(x), _bound_code(bound), float(eb), x.numel(), _ptr(x).value,
                                 _ptr(q.bins).value, _ptr(q.mask).value, _ptr(q.outliers).value,
                                 q.outliers.numel(), _ptr(q.header).value)
        self.items = items
        L = lib()
        self.plan = torch.empty(int(L.lcq_batch_plan_size(n)), dtype=torch.uint8, device=self.device)
        self.ws = torch.empty(int(L.lcq_batch_workspace_size(items, n)), dtype=torch.uint8,
                              device=self.device)
        self.info = BatchInfo()
        code = L.lcq_batch_prepare(items, n, _ptr(self.plan), self.plan.numel(), _ptr(self.ws),
                                   self.ws.numel(), ctypes.byref(self.info),
                                   _stream_ptr(stream, self.device))
        if code != 0:
            raise LcqError(code, "lcq_batch_prepare (item %d)" % self.info.bad_item)

    def run(self, stream=None):
        code = lib().lcq_quantize_batched(ctypes.byref(self.info), _ptr(self.plan), _ptr(self.ws),
                                          self.ws.numel(), _stream_ptr(stream, self.device))
        _check(code, "lcq_quantize_batched")

    def autotune(self, reps=3, stream=None):
        nv = int(lib().lcq_batch_tune_variant_count())
        ms = (ctypes.c_float * nv)()
        code = lib().lcq_autotune_batched(ctypes.byref(self.info), _ptr(self.plan), _ptr(self.ws),
                                          self.ws.numel(), _stream_ptr(stream, self.device), int(reps), ms)
        _check(code, "lcq_autotune_batched")
        return list(ms)


def batch_variant_count():
    return int(lib().lcq_batch_tune_variant_count())


def set_batch_variant(v):
    _check(lib().lcq_batch_tune_set(int(v)), "lcq_batch_tune_set")


def get_batch_variant():
    return int(lib().lcq_batch_tune_get())


def fp64_mul_rate(device, ctas_per_sm=8, iters=1 << 14, reps=5):
    """Float64 multiplications per second of this GPU, measured by
    lcq_probe_fp64_mul with CUDA events (best of `reps` launches)."""
    sink = torch.empty(1, dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream(device)
    cnt = _u64(0)
    _check(lib().lcq_probe_fp64_mul(ctas_per_sm, iters, _ptr(sink), ctypes.byref(cnt), _vp(stream.cuda_stream)),
           "lcq_probe_fp64_mul")
    best = None
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        _check(lib().lcq_probe_fp64_mul(ctas_per_sm, iters, _ptr(sink), None, _vp(stream.cuda_stream)),
               "lcq_probe_fp64_mul")
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b)
        best = ms if best is None else min(best, ms)
    return cnt.value / (best / 1e3)


def debug_set_scan(spin_limit=0, drop_tile=(1 << 64) - 1):
    """Test hook for the bounded scan waits (see include/lcq.h)."""
    lib().lcq_debug_set_scan(int(spin_limit), int(drop_tile))


def host_stage_size(dtype_code, n, cap):
    return int(lib().lcq_host_stage_size(dtype_code, int(n), int(cap)))


def quantize_host(x_host, bound, eb, outputs, stage, ws, stream=None, device=None):
    """End-to-end quantization of a (preferably pinned) host tensor through
    lcq_quantize_host: H2D copy, kernels, D2H copies of bins, mask, header and
    outliers into the host tensors of `outputs`.  Blocks until done."""
    device = device or torch.device("cuda", torch.cuda.current_device())
    code = lib().lcq_quantize_host(
        _dtype_code(x_host), _bound_code(bound), float(eb), _ptr(x_host), x_host.numel(),
        _ptr(outputs.bins), _ptr(outputs.mask), _ptr(outputs.outliers), outputs.outliers.numel(),
        _ptr(outputs.header), _ptr(stage), stage.numel(), _ptr(ws), ws.numel(),
        _stream_ptr(stream, device))
    _check(code, "lcq_quantize_host")
    return outputs


def host_items(jobs):
    """ctypes array of lcq_host_item from (x_host, bound, eb, outputs) tuples."""
    arr = (HostItem * len(jobs))()
    for it, (x, bound, eb, o) in zip(arr, jobs):
        it.dtype, it.bound_type, it.eb = _dtype_code(x), _bound_code(bound), float(eb)
        it.h_in, it.n = _ptr(x).value, x.numel()
        it.h_bins, it.h_mask, it.h_outliers = _ptr(o.bins).value, _ptr(o.mask).value, _ptr(o.outliers).value
        it.outlier_capacity = o.outliers.numel()
        it.h_hdr = _ptr(o.header).value
    return arr


def host_batch_stage_size(items):
    return int(lib().lcq_host_batch_stage_size(ctypes.cast(items, _vp), len(items)))


def quantize_host_batch(items, stage, ws, stream=None, device=None):
    """lcq_quantize_host_batch over a host_items() array; blocks until all
    results are on the host.  Returns the per-item status codes."""
    device = device or torch.device("cuda", torch.cuda.current_device())
    code = lib().lcq_quantize_host_batch(ctypes.cast(items, _vp), len(items), _ptr(stage), stage.numel(), _ptr(ws),
                                         ws.numel(), _stream_ptr(stream, device))
    _check(code, "lcq_quantize_host_batch")
    return [it.status for it in items]


def pack(codes, out=None, ws=None, stream=None):
    """Bit-plane packing of an int32 CUDA tensor (lcq_pack).  Returns (buffer,
    size tensor): the packed bytes are buffer[:size] (size is a device int64,
    no host synchronisation)."""
    _require_cuda(codes)
    n = codes.numel()
    if out is None:
        out = torch.empty(int(lib().lcq_pack_bound(n)), dtype=torch.uint8, device=codes.device)
    if ws is None:
        ws = torch.empty(max(int(lib().lcq_pack_workspace_size(n)), 16), dtype=torch.uint8, device=codes.device)
    size = torch.empty(1, dtype=torch.int64, device=codes.device)
    code = lib().lcq_pack(_ptr(codes), n, _ptr(out), out.numel(), _ptr(size), _ptr(ws), ws.numel(),
                          _stream_ptr(stream, codes.device))
    _check(code, "lcq_pack")
    return out, size


def unpack(buf, n, ws=None, stream=None, check=True):
    """Codes back from a packed buffer (uint8 CUDA tensor of its bytes)."""
    _require_cuda(buf)
    codes = torch.empty(n, dtype=torch.int32, device=buf.device)
    if ws is None:
        ws = torch.empty(max(int(lib().lcq_pack_workspace_size(n)), 16), dtype=torch.uint8, device=buf.device)
    status = torch.zeros(1, dtype=torch.int32, device=buf.device)
    code = lib().lcq_unpack(_ptr(buf), buf.numel(), n, _ptr(codes), _ptr(status), _ptr(ws), ws.numel(),
                            _stream_ptr(stream, buf.device))
    _check(code, "lcq_unpack")
    if check and int(status.item()):
        raise LcqError(7, "lcq_unpack (device status %d)" % int(status.item()))
    return codes
