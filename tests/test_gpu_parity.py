"""CUDA path vs oracle, bit for bit: bins, outlier mask, outlier payload,
outlier count, header constants and decoded values (the quantities are exact,
so no tolerance applies).  Sizes span several 4096-value tiles and ragged
tails; the large cases use the benchmark's full configurations."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2407_15037_b300 as P
import synth
from gpu_helpers import compare

pytestmark = pytest.mark.gpu

DEV = "cuda"
BOUNDS = ["abs", "rel", "noa"]
EBS = [1e-2, 1e-3, 1e-4, 1e-5]


@pytest.fixture(autouse=True)
def _reset_scan():
    P.debug_set_scan(0)
    yield
    P.debug_set_scan(0)


def test_sine_1d_abs_config():
    """2^20 float32 sine + noise with 0.1% specials and bin-edge values, ABS 1e-3."""
    x = synth.sine_1d(1 << 20, seed=0, eb=1e-3, device=DEV)
    q, oq = compare(x, "abs", 1e-3)
    assert oq.count >= 1049 * 5 // 8  # NaN/Inf kinds are always outliers


@pytest.mark.parametrize("bound", BOUNDS)
@pytest.mark.parametrize("eb", EBS)
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_smooth_field_sweep(bound, eb, dtype):
    x = synth.smooth_field((37, 61, 53), dtype=dtype, seed=1, device=DEV)  # 119,561 values
    compare(x, bound, eb)


@pytest.mark.parametrize("n", [0, 1, 3, 4, 5, 31, 32, 33, 127, 4095, 4096, 4097, 8193, 12289, 65537])
@pytest.mark.parametrize("bound", BOUNDS)
def test_ragged_sizes(n, bound):
    g = torch.Generator(device=DEV).manual_seed(n)
    x = torch.randn(n, generator=g, device=DEV) * 10
    if n > 3:
        x[::7] = float("nan")
    compare(x, bound, 1e-3)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("bound", BOUNDS)
def test_special_values(dtype, bound):
    if dtype == torch.float32:
        bits = np.array([0x7FC00000, 0x7F800001, 0xFFC01234, 0x7F800000, 0xFF800000, 0, 0x80000000,
                         1, 0x807FFFFF, 0x7F7FFFFF, 0xFF7FFFFF, 0x00800000, 0x3F800000, 0xC0490FDB],
                        dtype=np.uint32)
        x = torch.from_numpy(np.tile(bits, 700).view(np.float32)).to(DEV)
    else:
        bits = np.array([0x7FF8000000000000, 0x7FF0000000000001, 0xFFF0000000000000, 0,
                         0x8000000000000000, 1, 0x800FFFFFFFFFFFFF, 0x7FEFFFFFFFFFFFFF,
                         0x0010000000000000, 0x3FF0000000000000], dtype=np.uint64)
        x = torch.from_numpy(np.tile(bits, 900).view(np.float64)).to(DEV)
    compare(x, bound, 1e-3)


def test_int_min_and_maxbin_edges():
    eb = 2.0 ** -10
    v = np.array([(2.0 ** 30 - 64) * 2 * eb, 2.0 ** 30 * 2 * eb, -(2.0 ** 30) * 2 * eb,
                  -(2.0 ** 31) * 2 * eb, 2.0 ** 31 * 2 * eb, -(2.0 ** 30 - 64) * 2 * eb],
                 dtype=np.float32)
    x = torch.from_numpy(np.tile(v, 1000)).to(DEV)
    q, oq = compare(x, "abs", eb)
    assert oq.count == 4000


@pytest.mark.parametrize("eb", [1e-3, 1e-6])
def test_rel_stress_subset(eb):
    x = synth.rel_stress(1 << 22, seed=0, device=DEV)
    q, oq = compare(x, "rel", eb)
    assert oq.count >= 0.111 * x.numel()


def test_noa_degenerate_all_outliers():
    x = torch.full((10000,), 2.5, device=DEV)
    q, oq = compare(x, "noa", 1e-3)
    assert oq.count == 10000
    x = torch.full((5000,), float("nan"), device=DEV)
    compare(x, "noa", 1e-3)
    # only signed zeros: a zero range is +0 in the header on both sides
    x = torch.zeros(3000, device=DEV)
    x[::3] = -0.0
    compare(x, "noa", 1e-3)
    compare(torch.full((70,), -0.0, dtype=torch.float64, device=DEV), "noa", 1e-3)


def test_capacity_overflow_reports_and_stays_in_bounds():
    x = torch.full((50000,), float("inf"), device=DEV)
    cap = 1000
    q = P.alloc_outputs(x.numel(), x.dtype, x.device, outlier_capacity=cap + 64)
    guard = q.outliers[cap:].clone().fill_(0x5A5A5A5A)
    q.outliers[cap:] = guard
    small = P.Quantized(q.bins, q.mask, q.outliers[:cap], q.header, q.n, q.dtype)
    ws = P.new_workspace(x.numel(), x.device)
    P.quantize_into(x, "abs", 1e-3, small, ws)
    code, cnt = P.sync_status(small)
    assert code == 3 and cnt == 50000  # LCQ_ERR_CAPACITY, full count
    assert torch.equal(q.outliers[cap:], guard)  # nothing written past the capacity
    compare(x, "abs", 1e-3, q=small, capacity=cap, check_decode=False)


def test_bad_bounds_rejected():
    x = torch.randn(100, device=DEV)
    for eb in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(P.LcqError):
            P.quantize(x, "abs", eb)
    with pytest.raises(P.LcqError):
        P.quantize(x, "rel", 1e-46)


def test_workspace_reuse_across_calls():
    ws = P.new_workspace(1 << 20, DEV)
    for i, n in enumerate([1 << 20, 5000, 1 << 18, 77777, 1 << 20]):
        g = torch.Generator(device=DEV).manual_seed(i)
        x = torch.randn(n, generator=g, device=DEV) * 100
        bound = BOUNDS[i % 3]
        q = P.alloc_outputs(n, x.dtype, x.device)
        P.quantize_into(x, bound, 1e-4, q, ws)
        compare(x, bound, 1e-4, q=q)


def test_workspace_shared_by_arrays_of_different_sizes():
    """One workspace sized for the largest array serves quantize and
    dequantize calls on arrays of several sizes in turn (a large array's
    tile table covers the place where a small array's would lie): every
    result, encoded and decoded with that workspace, equals the oracle's."""
    sizes = [1 << 24, 300007, 1 << 24, 5000, (1 << 22) + 3]
    ws = P.new_workspace(1 << 24, DEV)
    for i, n in enumerate(sizes):
        x = synth.smooth_field((n,), dtype=torch.float32, seed=40 + i, device=DEV)
        for bound, eb in (("abs", 1e-5), ("rel", 1e-4), ("noa", 1e-5)):
            q = P.alloc_outputs(n, x.dtype, x.device)
            P.quantize_into(x, bound, eb, q, ws)
            xr = torch.empty_like(x)
            P.lcq.dequantize_into(q, xr, ws)
            _, oq = compare(x, bound, eb, q=q, check_decode=False)
            assert oq.count > 0
            assert np.array_equal(xr.cpu().numpy().view(np.uint32), O.dequantize(oq).view(np.uint32))


def test_scan_timeout_is_reported_without_hang():
    """A bounded wait that runs out: with the test hook, the quantize kernel's
    scan warp never hands scan tile 1 back to its compute warps; their wait
    gives up after the poll limit, the kernel finishes, and the call reports
    LCQ_STATUS_TIMEOUT.  After the workspace is zeroed the same call is exact."""
    x = torch.randn(1 << 19, device=DEV)  # several scan tiles of every tile shape
    ws = P.new_workspace(x.numel(), x.device)
    q = P.alloc_outputs(x.numel(), x.dtype, x.device)
    P.debug_set_scan(spin_limit=200, drop_tile=1)
    try:
        P.quantize_into(x, "abs", 1e-3, q, ws)
        code, _ = P.sync_status(q)
    finally:
        P.debug_set_scan(0)
    assert code == 4  # LCQ_ERR_TIMEOUT
    ws.zero_()
    P.quantize_into(x, "abs", 1e-3, q, ws)
    assert P.sync_status(q)[0] == 0
    compare(x, "abs", 1e-3, q=q)


def test_dequantize_rejects_mismatched_header():
    x = torch.randn(10000, device=DEV)
    q = P.quantize(x, "abs", 1e-3)
    out = torch.full((10000,), 7.0, device=DEV)
    status = torch.zeros(1, dtype=torch.int32, device=DEV)
    ws = P.new_workspace(10000, DEV)
    wrong = P.Quantized(q.bins[:9000], q.mask[:282], q.outliers, q.header, 9000, q.dtype)
    P.dequantize_into(wrong, out[:9000], ws, status)
    torch.cuda.synchronize()
    assert int(status.item()) & P.lcq.STATUS_HEADER
    assert torch.all(out == 7.0)


@pytest.mark.parametrize("bound", BOUNDS)
@pytest.mark.parametrize("dtype,n", [(torch.float32, 64 ** 3), (torch.float32, 3 * (1 << 23) + 12345),
                                     (torch.float64, (1 << 23) + 77)])
def test_host_entry_point_matches_device_path(bound, dtype, n):
    """lcq_quantize_host (host buffers; the input goes up and the results come
    down in pipelined chunks of 2^23 values) gives exactly what the device
    entry point gives: one partial chunk, several chunks with a ragged tail,
    float64, and outliers spread over every chunk."""
    x = synth.smooth_field((n,), dtype=dtype, seed=3, device=DEV)
    x[::4099] = float("nan")
    xp = x.cpu().pin_memory()
    idt = torch.int32 if dtype == torch.float32 else torch.int64
    outs = P.Quantized(torch.empty(n, dtype=torch.int32).pin_memory(),
                       torch.empty((n + 31) // 32, dtype=torch.int32).pin_memory(),
                       torch.empty(n, dtype=idt).pin_memory(),
                       torch.empty(P.lcq.HEADER_BYTES, dtype=torch.uint8).pin_memory(), n, dtype)
    dc = P.lcq._dtype_code(x)
    stage = torch.empty(P.host_stage_size(dc, n, n), dtype=torch.uint8, device=DEV)
    ws = P.new_workspace(n, DEV)
    P.quantize_host(xp, bound, 1e-4, outs, stage, ws)
    qd = P.quantize(x, bound, 1e-4)
    torch.cuda.synchronize()
    h = qd.read_header()
    assert h.outlier_count >= n // 4099
    assert torch.equal(outs.bins, qd.bins.cpu())
    assert torch.equal(outs.mask, qd.mask.cpu())
    assert torch.equal(outs.outliers[:h.outlier_count], qd.outliers[:h.outlier_count].cpu())
    assert torch.equal(outs.header, qd.header.cpu())


def test_host_batch_matches_device_path():
    """lcq_quantize_host_batch: items of both data types, all bound types,
    one and several chunks, pipelined over two stage slots; every item gives
    exactly what the device entry point gives, with its status."""
    specs = [(torch.float32, "abs", 3 * (1 << 23) + 999), (torch.float64, "rel", 70001),
             (torch.float32, "noa", (1 << 23) + 32), (torch.float32, "rel", 4096),
             (torch.float64, "noa", (1 << 23) + 5), (torch.float32, "abs", 1)]
    jobs, refs = [], []
    for k, (dt, bound, n) in enumerate(specs):
        x = synth.smooth_field((n,), dtype=dt, seed=10 + k, device=DEV)
        x[::3001] = float("nan")
        xp = x.cpu().pin_memory()
        idt = torch.int32 if dt == torch.float32 else torch.int64
        outs = P.Quantized(torch.empty(n, dtype=torch.int32).pin_memory(),
                           torch.empty((n + 31) // 32, dtype=torch.int32).pin_memory(),
                           torch.empty(n, dtype=idt).pin_memory(),
                           torch.empty(P.lcq.HEADER_BYTES, dtype=torch.uint8).pin_memory(), n, dt)
        jobs.append((xp, bound, 1e-4, outs))
        refs.append(P.quantize(x, bound, 1e-4))
    items = P.lcq.host_items(jobs)
    stage = torch.empty(P.lcq.host_batch_stage_size(items), dtype=torch.uint8, device=DEV)
    ws = P.new_workspace(max(n for _, _, n in specs), DEV)
    assert P.lcq.quantize_host_batch(items, stage, ws) == [0] * len(specs)
    torch.cuda.synchronize()
    for (xp, bound, eb, outs), qd in zip(jobs, refs):
        h = qd.read_header()
        assert torch.equal(outs.bins, qd.bins.cpu())
        assert torch.equal(outs.mask, qd.mask.cpu())
        assert torch.equal(outs.outliers[:h.outlier_count], qd.outliers[:h.outlier_count].cpu())
        assert torch.equal(outs.header, qd.header.cpu())


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_every_tile_shape_variant_matches_oracle(dtype):
    """Every tile shape the autotuner may pick gives the same bits."""
    x = synth.smooth_field((71, 67, 59), dtype=dtype, seed=5, device=DEV)  # ragged: 280,663 values
    x[::1001] = float("nan")
    dc = P.lcq._dtype_code(x)
    saved = [P.lcq.get_variant(0, dc, b) for b in BOUNDS] + [P.lcq.get_variant(1, dc, "abs")]
    try:
        for v in range(P.lcq.variant_count()):
            for bound in BOUNDS:
                P.lcq.set_variant(0, P.lcq._dtype_code(x), bound, v)
            P.lcq.set_variant(1, P.lcq._dtype_code(x), "abs", v)
            for bound in BOUNDS:
                compare(x, bound, 1e-4)
    finally:
        for bound, v in zip(BOUNDS, saved):
            P.lcq.set_variant(0, dc, bound, v)
        P.lcq.set_variant(1, dc, "abs", saved[3])


def _f64_edge_values(rng, eb):
    eb2 = 2 * eb
    k = rng.integers(-(1 << 29), 1 << 29, 20000).astype(np.float64)
    edges = (k + 0.5) * eb2
    ulp = np.spacing(np.abs(edges))
    vals = [edges, edges + ulp, edges - ulp, edges + 2 * ulp, -edges]
    p2 = np.ldexp(1.0, rng.integers(-1022, 1023, 20000))
    vals += [p2, np.nextafter(p2, 0), np.nextafter(p2, np.inf), -p2]
    tiny = np.ldexp(1.0 + rng.random(20000), rng.integers(-1022, -500, 20000))  # around the 2^-511 rescale
    vals += [tiny, np.nextafter(np.ldexp(1.0, -1022), 0) * rng.random(2000)]    # and below the normals
    return np.concatenate(vals)


@pytest.mark.parametrize("bound", BOUNDS)
@pytest.mark.parametrize("eb", [1e-3, 1e-7])
def test_f64_random_bit_patterns_and_edges(bound, eb):
    """float64 over every exponent: random 64-bit patterns, a band of moderate
    magnitudes, and structured edges; the float64 recipes work on the bit
    patterns, so this exercises every branch of them."""
    rng = np.random.default_rng(int(-np.log10(eb)) * 7 + len(bound))
    raw = rng.integers(0, np.iinfo(np.uint64).max, 1 << 21, dtype=np.uint64, endpoint=True).view(np.float64)
    mod = rng.normal(0, 1, 1 << 21) * 10.0 ** rng.integers(-12, 12, 1 << 21)
    x = np.concatenate([raw, mod, _f64_edge_values(rng, eb)])
    compare(torch.from_numpy(x).to(DEV), bound, eb)


@pytest.mark.parametrize("bound", ["abs", "noa"])
@pytest.mark.parametrize("eb", [1e-3, 0.37, 1e300])
def test_f64_values_near_the_check_threshold(bound, eb):
    """float64 ABS / NOA skip the double-check where its outcome is certain
    (|q - b| <= 1/2 - 2^-20, |x| < 2^1022); values just inside and outside
    that margin, at bin edges of small and large bins, and near DBL_MAX
    (where b eb2 can overflow) must still match the oracle."""
    if bound == "noa" and eb == 1e300:
        pytest.skip("NOA bound is relative to the range")
    rng = np.random.default_rng(int(eb * 1000) % 97)
    eb2 = 2 * eb
    vals = []
    for k in (rng.integers(-(1 << 29), 1 << 29, 4000), rng.integers(-40, 40, 4000)):
        k = k.astype(np.float64)
        for f in (0.25, 0.5, 0.99, 1.0, 1.01, 2.0, 4.0, 64.0):
            for sgn in (-1.0, 1.0):
                with np.errstate(over="ignore"):  # beyond DBL_MAX: +-Inf, an outlier on both sides
                    vals.append((k + 0.5 + sgn * f * 2.0 ** -20) * eb2)
    big = np.finfo(np.float64).max * (1.0 - rng.random(20000) * 1e-6)
    vals += [big, -big, np.ldexp(1.0 + rng.random(20000), 1022), np.ldexp(1.0 + rng.random(20000), 1021)]
    x = np.concatenate(vals)
    compare(torch.from_numpy(x).to(DEV), bound, eb)


@pytest.mark.parametrize("eb", [1e-2, 1e-3, 1e-5, 1e-6, 1e-7])
def test_f64_rel_values_near_the_binade_margin(eb):
    """float64 REL skips the rest of its check where the reconstruction
    provably stays in the value's binade and passes (mantissa at least
    step/2 + 2^-40 inside the binade, exponent high enough); values on both
    sides of that margin, at both ends of the binade, over a wide range of
    exponents (around 2^-511 and the smallest normals too) must still match
    the oracle, with the margin on (eb >= ~1e-6) and off (smaller eb)."""
    rng = np.random.default_rng(int(-np.log10(eb)))
    step = 2 * eb / (1 + eb)
    n = 6000
    f0 = step / 2 + 2.0 ** -40
    fr = []
    for d in (-4.0, -1.0, -2.0 ** -10, 0.0, 2.0 ** -10, 1.0, 4.0):
        off = d * 2.0 ** -40 + rng.random(n) * 2.0 ** -45
        fr += [f0 + off, 1.0 - f0 - off]
    fr.append(rng.random(n))
    f = np.clip(np.concatenate(fr), 0.0, np.nextafter(1.0, 0.0))
    e = np.concatenate([rng.integers(-1020, 1023, f.size // 2), rng.integers(-515, -505, f.size - f.size // 2)])
    x = np.ldexp(1.0 + f, e) * rng.choice([-1.0, 1.0], f.size)
    compare(torch.from_numpy(x).to(DEV), "rel", eb)


# --------------------------------------------------------- full sizes ----
# Every configuration the benchmark times, at its full size, compared over
# every value: the float32 512^3 and float64 256^3 fields at all four bounds
# of the sweep and all three bound types, and the 2^28-value REL stress input
# at both of its bounds, decoded values included.

@pytest.fixture(scope="module")
def field_f32_512():
    x = synth.smooth_field((512, 512, 512), dtype=torch.float32, seed=0, device=DEV)
    yield x
    del x
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def field_f64_256():
    x = synth.smooth_field((256, 256, 256), dtype=torch.float64, seed=0, device=DEV)
    yield x
    del x
    torch.cuda.empty_cache()


@pytest.mark.parametrize("eb", EBS)
@pytest.mark.parametrize("bound", BOUNDS)
def test_full_field_f32_512(field_f32_512, bound, eb):
    """The benchmark's workload: float32 512^3 sinusoid field, every bound
    type and bound of the timed sweep, compared over every value."""
    compare(field_f32_512, bound, eb)


@pytest.mark.parametrize("eb", EBS)
@pytest.mark.parametrize("bound", BOUNDS)
def test_full_field_f64_256(field_f64_256, bound, eb):
    compare(field_f64_256, bound, eb)


@pytest.mark.parametrize("eb", [1e-3, 1e-6])
def test_full_rel_stress_2_28(eb):
    x = synth.rel_stress(1 << 28, seed=0, device=DEV)
    compare(x, "rel", eb)
