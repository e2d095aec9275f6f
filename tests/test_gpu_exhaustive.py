"""All 2^32 float32 bit patterns through the CUDA path, compared with the
oracle bit for bit (the exhaustive run of Sec. 6, plus CPU/GPU parity of
Sec. 3.2).  ABS and REL run in chunks of 2^28 patterns (their constants do
not depend on the data) at two bounds, 1e-3 and 1e-5 (REL at 1e-5 has about
ten times the outliers of 1e-3 and other bin ranges); NOA runs as ONE call
over all 2^32 values, which also exercises the library's internal chunking
past 2^31 values."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2407_15037_b300 as P

pytestmark = pytest.mark.gpu

DEV = "cuda"
CH = 1 << 28
FULL = 1 << 32
FLT_MAX = float(np.finfo(np.float32).max)


def _patterns(start, count):
    return torch.arange(start, start + count, dtype=torch.int64, device=DEV).to(torch.int32).view(
        torch.float32)


def _check_chunk(c, xh, bins, mask, pay, base_count):
    oq = O.quantize_parallel(c, xh)
    assert np.array_equal(bins, oq.bins)
    assert np.array_equal(mask, oq.mask)
    assert np.array_equal(pay[base_count:base_count + oq.count], oq.payload)
    return oq.count


@pytest.mark.parametrize("eb", [1e-3, 1e-5])
@pytest.mark.parametrize("bound", ["abs", "rel"])
def test_all_patterns_chunked(bound, eb):
    c = O.consts(bound, np.float32, eb)
    ws = P.new_workspace(CH, DEV)
    q = P.alloc_outputs(CH, torch.float32, DEV)
    for start in range(0, FULL, CH):
        x = _patterns(start, CH)
        P.quantize_into(x, bound, eb, q, ws)
        h = q.read_header()
        assert h.status == 0
        xh = x.cpu().numpy()
        cnt = _check_chunk(c, xh, q.bins.cpu().numpy(), q.mask.cpu().numpy().view(np.uint32),
                           q.outliers[:h.outlier_count].cpu().numpy().view(np.uint32), 0)
        assert cnt == h.outlier_count
        # the decoded chunk stays within the bound (exact verifier)
        xr = P.dequantize(q, ws=ws).cpu().numpy()
        bad = O.verify_rel_parallel(xh, xr, eb) if bound == "rel" else O.verify_abs_parallel(xh, xr, eb)
        assert bad == 0


def test_all_patterns_noa_single_call():
    eb = 1e-3
    x = torch.arange(0, FULL, dtype=torch.int64, device=DEV).to(torch.int32).view(torch.float32)
    q = P.quantize(x, "noa", eb, outlier_capacity=1 << 26)
    h = q.read_header()
    assert h.status == 0 and h.mode == 0
    c = O.consts("noa", np.float32, eb, rng=(True, -FLT_MAX, FLT_MAX))
    assert h.range == c.R and h.eb_abs == c.eb_abs
    pay = q.outliers[:h.outlier_count].cpu().numpy().view(np.uint32)
    seen = 0
    for start in range(0, FULL, CH):
        xh = x[start:start + CH].cpu().numpy()
        seen += _check_chunk(c, xh, q.bins[start:start + CH].cpu().numpy(),
                             q.mask[start // 32:(start + CH) // 32].cpu().numpy().view(np.uint32),
                             pay, seen)
    assert seen == h.outlier_count
    del x
    xr = P.dequantize(q)
    torch.cuda.synchronize()
    for start in range(0, FULL, CH):
        xh = _patterns(start, CH).cpu().numpy()
        assert O.verify_abs_parallel(xh, xr[start:start + CH].cpu().numpy(), c.eb_abs) == 0
