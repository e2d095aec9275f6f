"""The 16-bit formats (IEEE binary16, bfloat16) on the CUDA path: bins, mask,
outlier payload, count and decoded values equal the oracle's bit for bit.

The oracle's 16-bit recipe (the float recipe on the widened value, checked
against the decoder's 16-bit rounding) is pinned in test_oracle_half.py.
Cases: every 16-bit pattern at several bounds of each type (also shuffled and
repeated over many tiles with a ragged tail, in both tile shapes), smooth
fields with a ragged length, the benchmark's 512^3 workload over every
value, the NOA range entry points, the host-buffer entry point over several
pipelined chunks, and the calls that refuse 16-bit data."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2407_15037_b300 as P
from paper_2407_15037_b300 import lcq as L
import synth

pytestmark = pytest.mark.gpu

DEV = "cuda"
FMTS = {"f16": torch.float16, "bf16": torch.bfloat16}
CODES = {"f16": 2, "bf16": 3}
ALL16 = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)


def _bits(t):
    return t.contiguous().view(torch.int16).cpu().numpy().view(np.uint16)


def _tensor(bits, fmt):
    return torch.from_numpy(bits.view(np.int16).copy()).view(FMTS[fmt]).to(DEV)


def _oracle(bits, bound, eb, fmt):
    x = bits.view(np.float16) if fmt == "f16" else bits
    return O.quantize(x, bound, eb, fmt=None if fmt == "f16" else "bf16")


def _compare(q, oq, fmt):
    h = q.read_header()
    assert h.status == 0 and h.dtype == CODES[fmt]
    assert h.outlier_count == oq.count
    assert np.array_equal(q.bins.cpu().numpy(), oq.bins)
    assert np.array_equal(q.mask.cpu().numpy().view(np.uint32), oq.mask)
    assert np.array_equal(_bits(q.outliers[:oq.count]), oq.payload)
    xr = P.dequantize(q)
    assert xr.dtype == FMTS[fmt]
    assert np.array_equal(_bits(xr), O.dequantize(oq).view(np.uint16))


EBS = [1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-8]


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("bound", ["abs", "rel", "noa"])
@pytest.mark.parametrize("eb", EBS)
def test_every_pattern(fmt, bound, eb):
    x = _tensor(ALL16, fmt)
    _compare(P.quantize(x, bound, eb), _oracle(ALL16, bound, eb, fmt), fmt)


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("bound", ["abs", "rel", "noa"])
def test_shuffled_patterns_over_many_tiles(fmt, variant, bound):
    rng = np.random.default_rng(CODES[fmt] * 10 + variant)
    bits = np.concatenate([rng.permutation(ALL16) for _ in range(5)] + [ALL16[rng.integers(0, 1 << 16, 77)]])
    code = CODES[fmt]
    saved = L.get_variant(0, code, bound)
    L.set_variant(0, code, bound, variant)
    try:
        q = P.quantize(_tensor(bits, fmt), bound, 1e-3)
        torch.cuda.synchronize()
    finally:
        L.set_variant(0, code, bound, saved)
    _compare(q, _oracle(bits, bound, 1e-3, fmt), fmt)


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("variant", [1, 5])
def test_dequantize_shapes(fmt, variant):
    rng = np.random.default_rng(7)
    bits = np.concatenate([rng.permutation(ALL16) for _ in range(3)] + [ALL16[:1001]])
    q = P.quantize(_tensor(bits, fmt), "rel", 1e-3)
    oq = _oracle(bits, "rel", 1e-3, fmt)
    code = CODES[fmt]
    saved = L.get_variant(1, code, 0)
    L.set_variant(1, code, 0, variant)
    try:
        xr = P.dequantize(q)
    finally:
        L.set_variant(1, code, 0, saved)
    assert np.array_equal(_bits(xr), O.dequantize(oq).view(np.uint16))


def test_tile_shapes_outside_the_16_bit_set_are_refused():
    for code in (2, 3):
        with pytest.raises(P.LcqError):
            L.set_variant(0, code, P.ABS, 3)
        with pytest.raises(P.LcqError):
            L.set_variant(1, code, 0, 2)


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("bound", ["abs", "rel", "noa"])
@pytest.mark.parametrize("eb", [1e-2, 1e-3, 1e-4])
def test_smooth_field_ragged(fmt, bound, eb):
    n = 1_000_003
    x = synth.smooth_field((n,), dtype=torch.float32, seed=5, device=DEV).to(FMTS[fmt])
    x[::9973] = float("nan")
    x[17::20011] = 0.0
    bits = _bits(x)
    _compare(P.quantize(x, bound, eb), _oracle(bits, bound, eb, fmt), fmt)


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_noa_range_entry_points(fmt):
    n = 300_001
    x = synth.smooth_field((n,), dtype=torch.float32, seed=8, device=DEV).to(FMTS[fmt])
    x[::1001] = float("inf")
    bits = _bits(x)
    xo = bits.view(np.float16) if fmt == "f16" else bits
    f = None if fmt == "f16" else "bf16"
    rng = O.value_range(xo, fmt=f)
    got = P.finite_range(x).cpu().numpy()
    assert bool(got[0]) == rng[0] and got[1] == rng[1] and got[2] == rng[2]
    q = P.alloc_outputs(n, x.dtype, DEV)
    ws = P.new_workspace(n, DEV)
    P.quantize_noa_range_into(x, 1e-3, rng, q, ws)
    _compare(q, O.quantize_with(O.consts("noa", fmt, 1e-3, rng=rng), xo), fmt)
    # a range value that is not a value of the format is refused
    with pytest.raises(P.LcqError):
        P.quantize_noa_range_into(x, 1e-3, (True, rng[1], rng[2] + 2.0 ** -30), q, ws)


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_noa_without_finite_values(fmt):
    bits = np.array([0x7C00, 0xFC00, 0x7E00] * 11 if fmt == "f16" else [0x7F80, 0xFF80, 0x7FC0] * 11, np.uint16)
    q = P.quantize(_tensor(bits, fmt), "noa", 1e-3)
    h = q.read_header()
    assert h.mode == 1 and h.outlier_count == bits.size
    _compare(q, _oracle(bits, "noa", 1e-3, fmt), fmt)


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
def test_host_entry_point_several_chunks(fmt):
    n = 2 * (1 << 23) + 999
    dt = FMTS[fmt]
    x = synth.smooth_field((n,), dtype=torch.float32, seed=4, device=DEV).to(dt)
    x[::4099] = float("nan")
    xp = x.cpu().pin_memory()
    outs = P.Quantized(torch.empty(n, dtype=torch.int32).pin_memory(),
                       torch.empty((n + 31) // 32, dtype=torch.int32).pin_memory(),
                       torch.empty(n, dtype=torch.int16).pin_memory(),
                       torch.empty(P.lcq.HEADER_BYTES, dtype=torch.uint8).pin_memory(), n, dt)
    stage = torch.empty(P.host_stage_size(CODES[fmt], n, n), dtype=torch.uint8, device=DEV)
    ws = P.new_workspace(n, DEV)
    P.quantize_host(xp, "abs", 1e-3, outs, stage, ws)
    qd = P.quantize(x, "abs", 1e-3)
    torch.cuda.synchronize()
    h = qd.read_header()
    assert h.outlier_count >= n // 4099
    assert torch.equal(outs.bins, qd.bins.cpu())
    assert torch.equal(outs.mask, qd.mask.cpu())
    assert torch.equal(outs.outliers[:h.outlier_count], qd.outliers[:h.outlier_count].cpu())
    assert torch.equal(outs.header, qd.header.cpu())
    oq = _oracle(_bits(x), "abs", 1e-3, fmt)
    assert np.array_equal(outs.bins.numpy(), oq.bins)


def test_calls_that_take_float_and_double_only():
    x = torch.zeros(4096, dtype=torch.float16, device=DEV)
    with pytest.raises(P.LcqError):
        L.quantize_ablation(x, "abs_no_check", 1e-3)
    q = P.quantize(x, "abs", 1e-3)
    # decoding as the other 16-bit format is refused by the header check
    out = torch.empty(4096, dtype=torch.bfloat16, device=DEV)
    ws = P.new_workspace(4096, DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    P.lcq.dequantize_into(q, out, ws, status)
    assert int(status.item()) & P.lcq.STATUS_HEADER


@pytest.mark.parametrize("fmt", ["f16", "bf16"])
@pytest.mark.parametrize("bound", ["abs", "rel", "noa"])
def test_full_field_512(fmt, bound):
    """The benchmark's 16-bit workload (the float32 512^3 field rounded to the
    format) at 1e-3, in the launch configuration the benchmark times,
    compared with the oracle over every value."""
    x = synth.smooth_field((512, 512, 512), dtype=torch.float32, seed=0, device=DEV).to(FMTS[fmt]).reshape(-1)
    q = P.quantize(x, bound, 1e-3)
    torch.cuda.synchronize()
    bits = _bits(x)
    xo = bits.view(np.float16) if fmt == "f16" else bits
    c = O.consts(bound, fmt, 1e-3, x=xo if bound == "noa" else None)
    _compare(q, O.quantize_parallel(c, xo), fmt)
