"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle on
the same input and compare every output bit for bit."""
import numpy as np
import torch

import oracle as O
import paper_2407_15037_b300 as P

UINT = {torch.float32: np.uint32, torch.float64: np.uint64}
NPF = {torch.float32: np.float32, torch.float64: np.float64}


def oracle_consts(bound, x_host, eb):
    return O.consts(bound, x_host.dtype, eb, x=x_host)


def compare(x, bound, eb, q=None, capacity=None, check_decode=True, oq=None):
    """Quantize device tensor x (unless q is given), quantize its host copy
    with the oracle, and assert equality of bins, mask, payload, count,
    header constants and decoded values.  Returns (q, oracle result)."""
    if q is None:
        q = P.quantize(x, bound, eb, outlier_capacity=capacity)
    torch.cuda.synchronize()
    h = q.read_header()
    xh = x.detach().cpu().numpy().reshape(-1)
    if oq is None:
        c = oracle_consts(bound, xh, eb)
        oq = O.quantize_parallel(c, xh) if capacity is None else O.quantize_with(c, xh, capacity)
    c = oq.consts
    u = UINT[x.dtype]
    f = NPF[x.dtype]
    assert h.magic == P.lcq.MAGIC
    assert h.n == xh.size
    assert h.outlier_count == oq.count, (h.outlier_count, oq.count)
    assert h.mode == c.all_outliers
    if not c.all_outliers:
        assert np.array(h.ebT_bits, dtype=np.uint64).astype(u).view(f) == f(c.ebT)
        scale = c.step if bound == "rel" else c.eb2
        inv = c.inv_l if bound == "rel" else c.inv
        assert np.array(h.scale_bits, dtype=np.uint64).astype(u).view(f) == f(scale)
        assert np.array(h.inv_bits, dtype=np.uint64).astype(u).view(f) == f(inv)
    if bound == "noa":
        bits = lambda v: np.float64(v).tobytes()
        assert bits(h.range) == bits(c.R) and bits(h.eb_abs) == bits(c.eb_abs)
    bins = q.bins.cpu().numpy()
    mismatch = np.flatnonzero(bins != oq.bins)
    assert mismatch.size == 0, "bins differ at %s" % mismatch[:10]
    assert np.array_equal(q.mask.cpu().numpy().view(np.uint32), oq.mask)
    cnt = min(oq.count, q.outliers.numel())
    pay = q.outliers[:cnt].cpu().numpy().view(u)
    assert np.array_equal(pay, oq.payload[:cnt])
    if check_decode and (capacity is None or oq.count <= capacity):
        xr = P.dequantize(q).cpu().numpy()
        oxr = O.dequantize(oq)
        assert np.array_equal(xr.view(u), oxr.view(u))
    return q, oq


CODES16 = {torch.float16: 2, torch.bfloat16: 3}


def bits16(t):
    return t.contiguous().view(torch.int16).cpu().numpy().view(np.uint16)


def compare16(x, bound, eb, q):
    """The 16-bit counterpart of compare: q (the CUDA path's result for the
    binary16 / bfloat16 tensor x) against the oracle's 16-bit recipe, bins,
    mask, payload, count and decoded values bit for bit."""
    torch.cuda.synchronize()
    bits = bits16(x).reshape(-1)
    xo = bits.view(np.float16) if x.dtype == torch.float16 else bits
    fmt = None if x.dtype == torch.float16 else "bf16"
    oq = O.quantize(xo, bound, eb, fmt=fmt)
    h = q.read_header()
    assert h.status == 0 and h.dtype == CODES16[x.dtype]
    assert h.outlier_count == oq.count
    assert np.array_equal(q.bins.cpu().numpy(), oq.bins)
    assert np.array_equal(q.mask.cpu().numpy().view(np.uint32), oq.mask)
    assert np.array_equal(bits16(q.outliers[:oq.count]), oq.payload)
    xr = P.dequantize(q)
    assert xr.dtype == x.dtype
    assert np.array_equal(bits16(xr), O.dequantize(oq).view(np.uint16))
    return q, oq
