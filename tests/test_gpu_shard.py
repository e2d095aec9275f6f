"""Sharded quantization on the CUDA path (one GPU, k shards of one array):
lcq_finite_range per shard equals the oracle's finite range; the combined
range fed to lcq_quantize_noa_range gives, per shard, exactly the unsharded
call's bins, mask words and outliers (at the exclusive-scan offsets), and the
same NOA constants; and the whole assembled result matches the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2407_15037_b300 as P
from paper_2407_15037_b300 import shard as S
import synth

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _bits(v):
    return np.float64(v).tobytes()


def _shard_run(x, eb, k):
    n = x.numel()
    bounds = [S.shard_bounds(n, k, r) for r in range(k)]
    ranges = []
    for a, b in bounds:
        r = P.finite_range(x[a:b]).cpu().tolist()
        got = (r[0] != 0.0, r[1], r[2])
        want = O.value_range(x[a:b].cpu().numpy())
        assert got[0] == want[0]
        if want[0]:
            assert got[1] == want[1] and got[2] == want[2]
        ranges.append(got)
    glob = S.combine_ranges(ranges)
    parts = []
    for a, b in bounds:
        xs = x[a:b]
        q = P.alloc_outputs(xs.numel(), x.dtype, DEV)
        ws = P.new_workspace(xs.numel(), DEV)
        P.quantize_noa_range_into(xs, eb, glob, q, ws)
        parts.append((a, b, q))
    return bounds, glob, parts


@pytest.mark.parametrize("k", [2, 3, 7])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_noa_shards_equal_unsharded(k, dtype):
    x = synth.smooth_field((45, 47, 49), dtype=dtype, seed=11, device=DEV).reshape(-1)
    x[::1013] = float("nan")
    x[7::2029] = float("-inf")
    eb = 1e-4
    whole = P.quantize(x, "noa", eb)
    hw = whole.read_header()
    _, glob, parts = _shard_run(x, eb, k)
    off = 0
    for a, b, q in parts:
        h = q.read_header()
        assert h.status == 0 and h.n == b - a
        for f in ("mode", "ebT_bits", "scale_bits", "inv_bits", "chk_bits"):
            assert getattr(h, f) == getattr(hw, f), f
        assert _bits(h.range) == _bits(hw.range) and _bits(h.eb_abs) == _bits(hw.eb_abs)
        assert torch.equal(q.bins, whole.bins[a:b])
        assert torch.equal(q.mask, whole.mask[a // 32:a // 32 + q.mask.numel()])
        assert torch.equal(q.outliers[:h.outlier_count], whole.outliers[off:off + h.outlier_count])
        off += h.outlier_count
    assert off == hw.outlier_count
    oq = O.quantize(x.cpu().numpy(), "noa", eb)
    assert oq.count == off and np.array_equal(whole.bins.cpu().numpy(), oq.bins)


def test_noa_shard_with_no_finite_value_and_empty_shard():
    x = synth.smooth_field((4099,), seed=3, device=DEV)
    x[:2080] = float("nan")  # shard 0 of 2 holds no finite value
    eb = 1e-3
    whole = P.quantize(x, "noa", eb)
    _, glob, parts = _shard_run(x, eb, 2)
    assert glob[0]
    assert torch.equal(torch.cat([q.bins for _, _, q in parts]), whole.bins)
    # n = 20 over 2 ranks: rank 1 is empty and still gets a complete header
    y = x[2080:2100].clone()
    _, glob, parts = _shard_run(y, eb, 2)
    (a0, b0, q0), (a1, b1, q1) = parts
    assert (a1, b1) == (20, 20)
    h1, h0 = q1.read_header(), q0.read_header()
    assert h1.magic == P.lcq.MAGIC and h1.n == 0 and h1.outlier_count == 0 and h1.status == 0
    assert h1.bound_type == P.NOA and h1.mode == h0.mode and h1.inv_bits == h0.inv_bits
    assert torch.equal(q0.bins, P.quantize(y, "noa", eb).bins)


def test_signed_zero_shards():
    x = torch.zeros(96, device=DEV)
    x[:64] = -0.0
    _, glob, parts = _shard_run(x, 1e-3, 2)
    whole = P.quantize(x, "noa", 1e-3).read_header()
    for _, _, q in parts:
        h = q.read_header()
        assert h.mode == 1 and _bits(h.range) == _bits(0.0) == _bits(whole.range)


@pytest.mark.parametrize("bound", ["abs", "rel", "noa"])
def test_quantize_sharded_single_rank_is_quantize(bound):
    x = synth.rel_stress(1 << 18, seed=4, device=DEV)
    r = S.quantize_sharded(x, bound, 1e-3)
    q = P.quantize(x, bound, 1e-3)
    h = q.read_header()
    assert r.offset == 0 and r.total == h.outlier_count
    assert torch.equal(r.q.bins, q.bins) and torch.equal(r.q.mask, q.mask)
    assert torch.equal(r.q.outliers[:r.total], q.outliers[:r.total])
