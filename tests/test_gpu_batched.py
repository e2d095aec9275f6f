"""Batched quantization (one header/range pass + one persistent launch over
many arrays of mixed size, dtype, bound type and bound): every array must
get exactly what lcq_quantize gives it alone, bit for bit, also when the
batch is captured in a CUDA graph and replayed, and for every tile-shape
variant; a sample of a batch shaped like the 4096-array workload is checked
against the oracle as well, and so is every array of a batch of binary16
and bfloat16 arrays."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2407_15037_b300 as P
import synth
from gpu_helpers import compare, compare16

pytestmark = pytest.mark.gpu

DEV = "cuda"


ALL_DTYPES = (torch.float32, torch.float64, torch.float16, torch.bfloat16)


def _mixed_arrays(seed=0, count=48, dtypes=ALL_DTYPES):
    rng = np.random.default_rng(seed)
    out = []
    sizes = [0, 1, 5, 33, 4095, 16384, 16385, 40000, 100003, 250000]
    for i in range(count):
        n = sizes[i % len(sizes)] if i < len(sizes) else int(rng.integers(1, 300000))
        dtype = dtypes[int(rng.integers(len(dtypes)))]
        bound = ("abs", "rel", "noa")[i % 3]
        eb = float(10 ** rng.uniform(-5, -2))
        src = dtype if dtype == torch.float64 else torch.float32
        x = synth.smooth_field((max(n, 1),), dtype=src, seed=seed * 1000 + i, device=DEV)[:n].to(dtype).contiguous()
        if n > 10 and i % 4 == 0:
            x[:: 9] = float("nan")
        if i == 11:
            x.fill_(3.0)  # NOA/ABS degenerate range
        out.append((x, bound, eb))
    return out


def _prepare(arrays):
    items = [(x, b, e, P.alloc_outputs(x.numel(), x.dtype, DEV)) for x, b, e in arrays]
    return P.Batch(items, DEV), items


def _check_against_single(items):
    torch.cuda.synchronize()
    for x, bound, eb, q in items:
        ref = P.quantize(x, bound, eb)
        torch.cuda.synchronize()
        assert bytes(q.header.cpu().numpy()) == bytes(ref.header.cpu().numpy()), (bound, x.numel())
        assert torch.equal(q.bins, ref.bins)
        assert torch.equal(q.mask, ref.mask)
        cnt = ref.read_header().outlier_count
        assert torch.equal(q.outliers[:cnt], ref.outliers[:cnt])


def test_batch_matches_single_array_calls():
    batch, items = _prepare(_mixed_arrays())
    batch.run()
    _check_against_single(items)


def test_batch_in_cuda_graph_replays():
    batch, items = _prepare(_mixed_arrays(seed=1))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        batch.run(stream=s)  # warm-up outside capture (first-use set-up)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        batch.run(stream=s)
    for _ in range(2):
        for _, _, _, q in items:
            q.bins.fill_(-7)
            q.mask.fill_(-7)
            q.header.fill_(0)
        g.replay()
        _check_against_single(items)


def test_every_batch_variant_matches():
    batch, items = _prepare(_mixed_arrays(seed=2, count=24))
    saved = P.lcq.get_batch_variant()
    try:
        for v in range(P.lcq.batch_variant_count()):
            P.lcq.set_batch_variant(v)
            for _, _, _, q in items:
                q.bins.fill_(-7)
            batch.run()
            _check_against_single(items)
    finally:
        P.lcq.set_batch_variant(saved)


def test_workload_shaped_batch_against_oracle():
    """4096 arrays with the workload's length, dtype, shape, bound-type and
    bound distributions, scaled to 2^27 values in total."""
    specs = synth.batch_specs(4096, seed=0, total_cap=1 << 27)
    arrays = [(synth.smooth_field(s["shape"], dtype=s["dtype"], seed=s["seed"], device=DEV),
               s["bound"], s["eb"]) for s in specs]
    batch, items = _prepare(arrays)
    batch.run()
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    for i in rng.choice(len(items), 24, replace=False):
        x, bound, eb, q = items[i]
        compare(x, bound, eb, q=q)
    # and every array against its single-array call
    _check_against_single(items[::16])


@pytest.mark.parametrize("dtype", [torch.float16, torch.bfloat16])
def test_16_bit_batch_against_oracle(dtype):
    """Ragged 16-bit arrays of every bound type, a whole 2^16-pattern sweep
    and an all-Inf/NaN NOA array among them, each against the oracle."""
    arrays = _mixed_arrays(seed=5, count=30, dtypes=(dtype,))
    pats = torch.from_numpy(np.arange(1 << 16, dtype=np.uint32).astype(np.uint16).view(np.int16).copy())
    sweep = pats.view(dtype).to(DEV)
    arrays += [(sweep, b, 1e-3) for b in ("abs", "rel", "noa")]
    arrays.append((torch.full((1000,), float("inf"), dtype=dtype, device=DEV), "noa", 1e-3))
    batch, items = _prepare(arrays)
    batch.run()
    for x, bound, eb, q in items:
        compare16(x, bound, eb, q)
    _check_against_single(items)


def test_batch_rejects_bad_items():
    x = torch.randn(1000, device=DEV)
    q = P.alloc_outputs(1000, x.dtype, DEV)
    with pytest.raises(P.LcqError):
        P.Batch([(x, "abs", 1e-3, q), (x, "abs", -1.0, q)], DEV)
    bad = x[1:]  # not 16-byte aligned
    with pytest.raises(P.LcqError):
        P.Batch([(x, "rel", 1e-3, q), (bad, "abs", 1e-3, P.alloc_outputs(999, x.dtype, DEV))], DEV)
