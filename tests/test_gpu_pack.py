"""The lossless stage on the CUDA path: lcq_pack gives byte for byte the
oracle's packed stream (and its size), lcq_unpack gives the codes back, over
ragged lengths, several chunks, extreme codes, and real bins and predictor
residuals; corrupted streams are reported, not over-read."""
import numpy as np
import pytest
import torch

import oracle.pack as PK
import paper_2407_15037_b300 as P
from paper_2407_15037_b300 import lcq as L
from paper_2407_15037_b300 import predictor as PD
import synth

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _check(codes_np):
    codes = torch.from_numpy(codes_np).to(DEV)
    buf, size = L.pack(codes)
    size = int(size.item())
    want = PK.pack(codes_np)
    assert size == len(want) == PK.packed_size(codes_np)
    assert bytes(buf[:size].cpu().numpy()) == want
    back = L.unpack(buf[:size].clone(), codes.numel())
    assert torch.equal(back, codes)


@pytest.mark.parametrize("n", [1, 31, 33, 8191, 8192, 8193, 70001])
def test_pack_matches_oracle(n):
    rng = np.random.default_rng(n)
    codes = rng.integers(-300, 300, n).astype(np.int32)
    codes[::97] = rng.integers(-2**31, 2**31, codes[::97].size, dtype=np.int64).astype(np.int32)
    codes[:1] = -2**31
    codes[n // 2: n // 2 + 64] = 0
    _check(codes)


def test_pack_quantizer_bins_and_residuals():
    N = 48
    x = synth.grf(N, seed=2, device=DEV)
    q = P.quantize(x, "abs", 1e-3)
    _check(q.bins.cpu().numpy())
    _check(PD.residuals(q.bins, N).cpu().numpy())


def test_pack_round_trip_large():
    n = (1 << 24) + 12345  # 2049 chunks
    g = torch.Generator(device=DEV).manual_seed(3)
    codes = (torch.randn(n, generator=g, device=DEV) * 1000).to(torch.int32)
    buf, size = L.pack(codes)
    size = int(size.item())
    assert torch.equal(L.unpack(buf[:size].clone(), n), codes)
    # the size is the sum of the block widths
    z = ((codes.to(torch.int64) << 1) ^ (codes.to(torch.int64) >> 63)) & 0xFFFFFFFF
    zp = torch.zeros(((n + 31) // 32) * 32, dtype=torch.int64, device=DEV)
    zp[:n] = z
    m = zp.view(-1, 32)
    acc = torch.zeros(m.shape[0], dtype=torch.int64, device=DEV)
    for i in range(32):
        acc |= m[:, i]
    w = torch.where(acc > 0, torch.floor(torch.log2(acc.double())).to(torch.int64) + 1, torch.zeros_like(acc))
    assert size == ((m.shape[0] + 15) // 16) * 16 + 4 * int(w.sum())


def test_corrupted_streams_are_reported():
    codes = torch.arange(-5000, 5000, dtype=torch.int32, device=DEV)
    buf, size = L.pack(codes)
    size = int(size.item())
    bad = buf[:size].clone()
    bad[0] = 200  # a width above 32
    with pytest.raises(P.LcqError):
        L.unpack(bad, codes.numel())
    with pytest.raises(P.LcqError):  # planes cut off
        L.unpack(buf[:size - 64].clone(), codes.numel())
