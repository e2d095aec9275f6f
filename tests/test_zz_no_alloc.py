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


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_noalloc_matches_lcq_quantize_on_two_calls(dtype):
    x = synth.smooth_field((101, 97, 89), dtype=dtype, seed=7, device=DEV)  # 871,933 values
    x[::997] = float("nan")
    n = x.numel()
    ws = P.new_workspace(n, DEV)
    for bound, eb in (("abs", 1e-4), ("rel", 1e-3), ("noa", 1e-5)):
        ref = P.quantize_into(x, bound, eb, P.alloc_outputs(n, dtype, DEV), ws)
        for _ in range(2):  # two calls in a row on the shared scratch
            got = P.alloc_outputs(n, dtype, DEV)
            assert _noalloc(x, bound, eb, got) == 0
            _same(got, ref)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = P.lib()
    too_big = int(L.lcq_noalloc_max_values()) + 1
    # rejected before anything is enqueued, so no buffers are needed
    code = L.lcq_quantize_noalloc(0, 0, 1e-3, None, too_big, None, None, None, 0, None,
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert code == 6  # LCQ_ERR_WORKSPACE
