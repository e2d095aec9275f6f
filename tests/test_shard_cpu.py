"""Shard invariance of the sharded protocol (NOA range all-reduce and the
exclusive scan of outlier counts, Sec. 2.1.3 over the union of shards).

Two gloo ranks run on the CPU.  Each quantizes its contiguous shard with the
oracle, using paper_2407_15037_b300.shard for everything that crosses ranks
(shard bounds, the range all-reduce, the payload offsets).  Rank 0 assembles
the shards and requires exactly the unsharded oracle result: bins, mask
words, payload, outlier count and the NOA constants.  Cases: ragged lengths,
a rank whose values are all NaN/Inf, an empty rank, a shard holding only
-0.0 against one holding +0.0, and ABS/REL (offsets only)."""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
import synth
from paper_2407_15037_b300 import shard as S

WORLD = 2


def _input(case):
    name, dtype, n = case[0], case[1], case[3]
    if name == "smooth":
        x = synth.smooth_field((n,), dtype=torch.float64, seed=5).numpy().astype(dtype)
        x[::997] = np.nan
        x[5::1999] = np.inf
        return x
    if name == "rank0_nonfinite":
        x = synth.smooth_field((n,), dtype=torch.float64, seed=6).numpy().astype(dtype)
        half = S.shard_bounds(n, WORLD, 0)[1]
        x[:half] = np.where(np.arange(half) % 2 == 0, np.nan, -np.inf)
        return x
    if name == "signed_zeros":
        x = np.zeros(n, dtype=dtype)
        x[: S.shard_bounds(n, WORLD, 0)[1]] = -0.0
        return x
    if name == "stress":
        return synth.rel_stress(n, seed=7).numpy().astype(dtype)
    raise KeyError(name)


# (input, dtype, bound, n, eb)
CASES = [
    ("smooth", np.float32, "noa", 100003, 1e-3),
    ("smooth", np.float64, "noa", 70001, 1e-6),
    ("rank0_nonfinite", np.float32, "noa", 4099, 1e-4),
    ("smooth", np.float32, "noa", 20, 1e-2),        # rank 1 holds nothing
    ("smooth", np.float32, "noa", 40, 1e-2),        # 32 + 8
    ("signed_zeros", np.float32, "noa", 96, 1e-3),  # range 0: every value an outlier
    ("stress", np.float32, "rel", 50000, 1e-3),
    ("stress", np.float64, "abs", 50000, 1e-9),
]


def _rank_main(rank, world, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for case in CASES:
            _run_case(rank, world, case)
    finally:
        dist.destroy_process_group()


def _run_case(rank, world, case):
    _, dtype, bound, n, eb = case
    x = _input(case)
    s0, s1 = S.shard_bounds(n, world, rank)
    xl = x[s0:s1]
    glob = None
    if bound == "noa":
        glob = S.allreduce_range(O.value_range(xl))
        c = O.consts("noa", dtype, eb, rng=glob)
    else:
        c = O.consts(bound, dtype, eb)
    oq = O.quantize_with(c, xl)
    off, total = S.exclusive_offsets(oq.count)
    parts = [None] * world
    dist.all_gather_object(parts, (s0, s1, off, total, oq.bins, oq.mask, oq.payload, glob))
    if rank != 0:
        return
    want = O.quantize(x, bound, eb)
    bins = np.empty(n, np.int32)
    mask = np.empty((n + 31) // 32, np.uint32)
    pay = np.empty(want.count, want.payload.dtype)
    for a, b, o, t, pb, pm, pp, g in parts:
        assert t == want.count, case
        assert g == glob, case
        bins[a:b] = pb
        mask[a // 32:a // 32 + pm.size] = pm
        pay[o:o + pp.size] = pp
    assert np.array_equal(bins, want.bins), case
    assert np.array_equal(mask, want.mask), case
    assert np.array_equal(pay.view(np.uint8), want.payload.view(np.uint8)), case
    if bound == "noa":
        wr = O.value_range(x)
        assert glob[0] == wr[0], case
        if wr[0]:
            assert (glob[1], glob[2]) == (wr[1], wr[2]), case
        assert np.float64(c.R).tobytes() == np.float64(want.consts.R).tobytes(), case
        assert c.eb_abs == want.consts.eb_abs and c.all_outliers == want.consts.all_outliers, case


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sharded_protocol_matches_unsharded_oracle_gloo():
    mp.start_processes(_rank_main, args=(WORLD, _free_port()), nprocs=WORLD, join=True, start_method="spawn")


@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 100, 4096, 100003])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_bounds_partition(n, world):
    prev = 0
    for r in range(world):
        a, b = S.shard_bounds(n, world, r)
        assert a == prev and a <= b
        assert (a % 32 == 0 or a == b == n) and (b % 32 == 0 or b == n)
        prev = b
    assert prev == n


def test_range_keys_order_and_round_trip():
    vals = [-math.inf, -1e308, -1.0, -5e-324, -0.0, 0.0, 5e-324, 1.0, 3.0, 1e308, math.inf]
    keys = [S.range_key(v) for v in vals]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    for v, k in zip(vals, keys):
        assert np.float64(S.range_unkey(k)).tobytes() == np.float64(v).tobytes()


def test_combine_ranges_matches_oracle_over_shards():
    rng = np.random.default_rng(3)
    x = rng.standard_normal(1000).astype(np.float32) * 100
    x[rng.integers(0, 1000, 50)] = np.nan
    x[:300] = np.inf
    parts = [O.value_range(x[a:b]) for a, b in ((0, 300), (300, 301), (301, 640), (640, 640), (640, 1000))]
    assert S.combine_ranges(parts) == O.value_range(x)
    assert S.combine_ranges([(False, 0.0, 0.0)] * 3) == (False, 0.0, 0.0)
    # signed zeros: -0.0 is the smaller key whichever shard holds it
    g = S.combine_ranges([(True, 0.0, 0.0), (True, -0.0, -0.0)])
    assert np.float64(g[1]).tobytes() == np.float64(-0.0).tobytes()
    assert np.float64(g[2]).tobytes() == np.float64(0.0).tobytes()
