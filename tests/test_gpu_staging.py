"""Float32 REL outlier staging: the quantize kernel copies each shared-memory
stage's outliers to a staging area and the compaction copies them to the
payload.  Every case is checked bit for bit against the oracle and against
the same call without staging (a workspace of the unstaged size), over every
tile shape: stages without outliers, sparse stages (staged), stages of
exactly half outliers (staged) and of one more (left to the compaction's
walk), fully dense stages, ragged tails, tiles that mix staged and unstaged
stages, a staging area that runs full, and a payload capacity that is too
small."""
import numpy as np
import pytest
import torch

import paper_2407_15037_b300 as P
import synth
from gpu_helpers import compare

pytestmark = pytest.mark.gpu

DEV = "cuda"
L = P.lcq


@pytest.fixture(autouse=True)
def _reset():
    saved = L.get_variant(0, L.F32, "rel")
    P.debug_set_scan(0)
    yield
    L.set_variant(0, L.F32, "rel", saved)
    P.debug_set_scan(0)


def _values(n, rng):
    """Nonzero normal float32 values over twelve decades, both signs."""
    mag = 10.0 ** rng.uniform(-6, 6, n)
    return (mag * np.where(rng.random(n) < 0.5, -1.0, 1.0)).astype(np.float32)


def _blocks(rng, block, counts, tail):
    """One block of `block` values per entry of counts, with that many REL
    outliers (zeros, NaN, Inf, denormals) at random places, then `tail`
    outlier-free values."""
    parts = []
    specials = np.array([0.0, -0.0, np.nan, np.inf, -np.inf, 1e-40], dtype=np.float32)
    for c in counts:
        v = _values(block, rng)
        if c:
            v[rng.choice(block, c, replace=False)] = rng.choice(specials, c)
        parts.append(v)
    parts.append(_values(tail, rng))
    return np.concatenate(parts)


def _unstaged(x, eb):
    n = x.numel()
    q = P.alloc_outputs(n, x.dtype, DEV)
    P.quantize_into(x, "rel", eb, q, P.new_workspace(n, DEV, L.F32, "abs"))
    return q


def _same(a, b):
    ha, hb = a.read_header(), b.read_header()
    assert ha.status == 0 and hb.status == 0
    assert ha.outlier_count == hb.outlier_count
    assert torch.equal(a.bins, b.bins) and torch.equal(a.mask, b.mask)
    assert torch.equal(a.outliers[:ha.outlier_count], b.outliers[:hb.outlier_count])


def test_staged_workspace_is_larger():
    n = 1 << 20
    assert P.workspace_size(L.F32, "rel", n) > P.workspace_size(L.F32, "abs", n)
    assert P.workspace_size(L.F64, "rel", n) == P.workspace_size(L.F64, "abs", n)


@pytest.mark.parametrize("variant", range(7))
def test_stage_densities_every_tile_shape(variant):
    """Blocks of 2048 values (a stage of the smallest shape; the larger
    stages cover two or four blocks) with outlier counts from none to all."""
    L.set_variant(0, L.F32, "rel", variant)
    rng = np.random.default_rng(100 + variant)
    pattern = [0, 1, 0, 200, 1024, 1025, 0, 2048, 0, 0, 0, 0, 7, 1500, 0, 0,
               0, 0, 0, 0, 0, 0, 0, 0, 31, 0, 0, 0, 2047, 0, 0, 0]
    counts = pattern * 3 + list(rng.integers(0, 300, 40))
    xh = _blocks(rng, 2048, counts, 1234)
    x = torch.from_numpy(xh).to(DEV)
    q, oq = compare(x, "rel", 1e-3)
    assert oq.count >= sum(counts)
    _same(q, _unstaged(x, 1e-3))


@pytest.mark.parametrize("variant", [0, 3, 4])
def test_staging_area_runs_full(variant):
    """About 40% outliers everywhere: every stage is below half, so each
    CTA's quarter share of the staging area fills and its later stages
    go to the compaction's walk."""
    L.set_variant(0, L.F32, "rel", variant)
    rng = np.random.default_rng(7 + variant)
    n = (1 << 21) + 777
    xh = _values(n, rng)
    xh[rng.random(n) < 0.4] = 0.0
    x = torch.from_numpy(xh).to(DEV)
    q, oq = compare(x, "rel", 1e-3)
    assert oq.count > n // 4  # more than the staging area holds
    _same(q, _unstaged(x, 1e-3))


def test_stress_input_small_bounds():
    """The REL stress recipe (magnitudes 10^U(-30, 30), zeros, denormals,
    NaN/Inf) at two bounds: 11% and 78% outliers."""
    x = synth.rel_stress((1 << 20) + 4321, seed=3, device=DEV)
    for eb in (1e-3, 1e-6):
        q, _ = compare(x, "rel", eb)
        _same(q, _unstaged(x, eb))


def test_staged_capacity_overflow():
    rng = np.random.default_rng(11)
    xh = _blocks(rng, 4096, [100] * 64, 999)
    x = torch.from_numpy(xh).to(DEV)
    cap = 3000
    q = P.alloc_outputs(x.numel(), x.dtype, DEV, outlier_capacity=cap + 64)
    guard = torch.full((64,), 0x5A5A5A5A, dtype=torch.int32, device=DEV)
    q.outliers[cap:] = guard
    small = P.Quantized(q.bins, q.mask, q.outliers[:cap], q.header, q.n, q.dtype)
    P.quantize_into(x, "rel", 1e-3, small, P.new_workspace(x.numel(), DEV))
    code, cnt = P.sync_status(small)
    assert code == 3 and cnt >= 6400
    assert torch.equal(q.outliers[cap:], guard)
    compare(x, "rel", 1e-3, q=small, capacity=cap, check_decode=False)
