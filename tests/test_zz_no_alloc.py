"""lcq_quantize_noalloc: the quantize entry point for callers that cannot
allocate device memory where they quantize (no-allocation regions such as a
fixed-budget streaming pipeline or a simulation step, or code running inside
another library's callback).  It takes no workspace; the library's built-in
device scratch array is used instead.

Called through the C ABI and compared with lcq_quantize on the same inputs,
bit for bit (the quantities are exact, so the tolerance is zero), on two
calls in a row, so that the second call runs on the scratch contents the
first one left behind.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import paper_2407_15037_b300 as P
import synth

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _noalloc(x, bound, eb, q):
    L = P.lib()
    code = L.lcq_quantize_noalloc(
        P.lcq._dtype_code(x), P.lcq._bound_code(bound), float(eb),
        ctypes.c_void_p(x.data_ptr()), x.numel(), ctypes.c_void_p(q.bins.data_ptr()),
        ctypes.c_void_p(q.mask.data_ptr()), ctypes.c_void_p(q.outliers.data_ptr()),
        q.outliers.numel(), ctypes.c_void_p(q.header.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return code


def _same(a, b):
    torch.cuda.synchronize()
    ha, hb = a.read_header(), b.read_header()
    assert ha.status == 0 and hb.status == 0
    assert bytes(a.header.cpu().numpy()) == bytes(b.header.cpu().numpy())
    assert torch.equal(a.bins, b.bins)
    assert torch.equal(a.mask, b.mask)
    cnt = ha.outlier_count
    assert torch.equal(a.outliers[:cnt], b.outliers[:cnt])


def _field(dtype):
    x = synth.smooth_field((101, 97, 89), dtype=torch.float64 if dtype == torch.float64 else torch.float32,
                           seed=7, device=DEV).to(dtype)  # 871,933 values
    x[::997] = float("nan")
    return x


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64, torch.float16, torch.bfloat16])
def test_noalloc_matches_lcq_quantize_on_two_calls(dtype):
    x = _field(dtype)
    n = x.numel()
    ws = P.new_workspace(n, DEV)
    for bound, eb in (("abs", 1e-4), ("rel", 1e-3), ("noa", 1e-5)):
        ref = P.quantize_into(x, bound, eb, P.alloc_outputs(n, dtype, DEV), ws)
        for _ in range(2):  # two calls in a row on the shared scratch
            got = P.alloc_outputs(n, dtype, DEV)
            assert _noalloc(x, bound, eb, got) == 0
            _same(got, ref)


def test_noalloc_call_after_a_timed_out_call_is_exact():
    """A call cut short leaves nothing behind for the next one: with the test
    hook, the quantize kernel's bounded wait for scan tile 1 runs out and the
    call reports a timeout; the next call on the same scratch, with the hook
    off, must give exactly what lcq_quantize gives."""
    x = _field(torch.float32)
    n = x.numel()
    ref = P.quantize_into(x, "abs", 1e-4, P.alloc_outputs(n, x.dtype, DEV), P.new_workspace(n, DEV))
    bad = P.alloc_outputs(n, x.dtype, DEV)
    P.debug_set_scan(spin_limit=200, drop_tile=1)
    try:
        assert _noalloc(x, "abs", 1e-4, bad) == 0
        code, _ = P.sync_status(bad)
    finally:
        P.debug_set_scan(0)
    assert code == 4  # LCQ_ERR_TIMEOUT
    for _ in range(2):
        got = P.alloc_outputs(n, x.dtype, DEV)
        assert _noalloc(x, "abs", 1e-4, got) == 0
        _same(got, ref)


def test_noalloc_rejected_call_enqueues_nothing():
    """Argument errors are reported before the shared scratch is touched; a
    valid call afterwards is exact."""
    x = _field(torch.float32)
    n = x.numel()
    q = P.alloc_outputs(n, x.dtype, DEV)
    assert _noalloc(x, "abs", -1.0, q) == 2       # LCQ_ERR_BOUND
    assert _noalloc(x, "abs", 1e-320, q) == 2     # ABS constants not normal
    L = P.lib()
    code = L.lcq_quantize_noalloc(0, 0, 1e-3, ctypes.c_void_p(x.data_ptr() + 4), n - 1,
                                  ctypes.c_void_p(q.bins.data_ptr()), ctypes.c_void_p(q.mask.data_ptr()),
                                  None, 0, ctypes.c_void_p(q.header.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 1  # LCQ_ERR_ARG: input not 16-byte aligned
    ref = P.quantize_into(x, "rel", 1e-3, P.alloc_outputs(n, x.dtype, DEV), P.new_workspace(n, DEV))
    assert _noalloc(x, "rel", 1e-3, q) == 0
    _same(q, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = P.lib()
    too_big = int(L.lcq_noalloc_max_values()) + 1
    # rejected before anything is enqueued, so no buffers are needed
    code = L.lcq_quantize_noalloc(0, 0, 1e-3, None, too_big, None, None, None, 0, None,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 6  # LCQ_ERR_WORKSPACE
