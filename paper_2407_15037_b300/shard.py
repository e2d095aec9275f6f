"""Sharded quantization of one array held by several ranks.

Each rank holds a contiguous index range of the array.  The per-value recipe
(Sec. 2.2-3.3) needs nothing from other ranks, so ABS and REL shards quantize
alone.  Two scalars do cross ranks:

* NOA (Sec. 2.1.3) bins against the range over the WHOLE array: one
  all-reduce combines every rank's finite minimum and maximum before binning.
* The outlier payload is kept in ascending index order over the whole array,
  so each rank's outliers start at the exclusive prefix sum of the counts of
  the ranks before it: one all-gather of one count.

With shard boundaries at multiples of 32 values every mask word belongs to
one rank, and the concatenation of the shards' bins, mask words and payloads
(at their offsets) is exactly the unsharded result.

The range is exchanged as order-preserving int64 keys of the float64 bit
patterns under a MIN reduction (the maximum as the complement of its key), so
the reduction is exact and independent of how a backend orders -0.0, +0.0
or compares floats.  The collectives are plain torch.distributed calls; with
no process group (or world size 1) the functions do no communication.
"""
from dataclasses import dataclass

import numpy as np
import torch
import torch.distributed as dist

from . import lcq as _L

_INT64_MAX = (1 << 63) - 1
_LOW63 = (1 << 63) - 1


def shard_bounds(n, world, rank, align=32):
    """[start, stop) of rank's contiguous shard of n values; boundaries are
    multiples of `align` (the last shard takes the ragged tail)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("shard_bounds: bad world/rank %r/%r" % (world, rank))
    units = (n + align - 1) // align
    per, extra = divmod(units, world)
    u0 = rank * per + min(rank, extra)
    u1 = u0 + per + (1 if rank < extra else 0)
    return min(n, u0 * align), min(n, u1 * align)


def range_key(v):
    """Order-preserving int64 key of a finite float64 value (-0.0 < +0.0)."""
    s = int(np.float64(v).view(np.int64))
    return s if s >= 0 else s ^ _LOW63


def range_unkey(k):
    s = k if k >= 0 else k ^ _LOW63
    return float(np.int64(s).view(np.float64))


def _keys(local):
    has, mn, mx = local
    if not has:
        return [_INT64_MAX, _INT64_MAX]
    return [range_key(mn), ~range_key(mx)]


def _from_keys(k0, k1):
    if k0 == _INT64_MAX:
        return (False, 0.0, 0.0)
    return (True, range_unkey(k0), range_unkey(~k1))


def combine_ranges(ranges):
    """Combination of several (has_finite, min, max) triples, exactly as
    allreduce_range combines them across ranks."""
    k0, k1 = _INT64_MAX, _INT64_MAX
    for r in ranges:
        a, b = _keys(r)
        k0, k1 = min(k0, a), min(k1, b)
    return _from_keys(k0, k1)


def _world(group):
    if group is None and not (dist.is_available() and dist.is_initialized()):
        return 1, 0
    return dist.get_world_size(group), dist.get_rank(group)


def _coll_device(group):
    if dist.get_backend(group) == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def allreduce_range(local, group=None):
    """Global (has_finite, min, max) from every rank's local triple: one
    all-reduce (MIN) of two int64 keys."""
    world, _ = _world(group)
    if world == 1:
        return combine_ranges([local])
    t = torch.tensor(_keys(local), dtype=torch.int64, device=_coll_device(group))
    dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
    k0, k1 = (int(v) for v in t.cpu().tolist())
    return _from_keys(k0, k1)


def exclusive_offsets(count, group=None):
    """(offset of this rank's outliers in the global payload, global count):
    one all-gather of one int64."""
    world, rank = _world(group)
    if world == 1:
        return 0, int(count)
    dev = _coll_device(group)
    mine = torch.tensor([int(count)], dtype=torch.int64, device=dev)
    parts = [torch.empty(1, dtype=torch.int64, device=dev) for _ in range(world)]
    dist.all_gather(parts, mine, group=group)
    counts = [int(p.item()) for p in parts]
    return sum(counts[:rank]), sum(counts)


@dataclass
class ShardResult:
    q: "_L.Quantized"   # this rank's bins, mask words, outliers (local order) and header
    offset: int         # index of this rank's first outlier in the global payload
    total: int          # outliers over all ranks
    range: tuple        # NOA: the global (has_finite, min, max); else None


def quantize_sharded(x_local, bound, eb, group=None, outlier_capacity=None, ws=None, stream=None):
    """Quantize this rank's shard (a contiguous CUDA tensor; every shard but
    the last a multiple of 32 values long) as part of the whole array.

    NOA: lcq_finite_range on the shard, allreduce_range, then
    lcq_quantize_noa_range with the global range.  Then the exclusive offsets
    of the outlier counts.  Both exchanges read a scalar result back to the
    host (they synchronise the stream)."""
    x = x_local.contiguous().reshape(-1)
    b = _L._bound_code(bound)
    q = _L.alloc_outputs(x.numel(), x.dtype, x.device, outlier_capacity)
    if ws is None:
        ws = _L.new_workspace(x.numel(), x.device, _L._dtype_code(x), b)
    rng = None
    if b == _L.NOA:
        r = _L.finite_range(x, ws, stream).cpu().tolist()
        rng = allreduce_range((r[0] != 0.0, r[1], r[2]), group)
        _L.quantize_noa_range_into(x, eb, rng, q, ws, stream)
    else:
        _L.quantize_into(x, b, eb, q, ws, stream)
    code, count = _L.sync_status(q, stream)
    _L._check(code, "quantize_sharded")
    offset, total = exclusive_offsets(count, group)
    return ShardResult(q, offset, total, rng)
