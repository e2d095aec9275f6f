"""Benchmark of the guaranteed-error-bound quantizers on B300.

One step = the quantize+verify sweep on the float32 512^3 sinusoid field
(sum of 8 random 3-D sinusoids + N(0, 0.01)): ABS, REL and NOA at bounds 1e-2,
1e-3, 1e-4 and 1e-5, i.e. 12 lcq_quantize calls (12 quantize kernels and 4
NOA range kernels), outlier compaction included.  Throughput is input bytes
per second (the paper's convention, Sec. 5), inputs resident in HBM; the
input (512 MiB) is larger than L2 (126 MB), so no L2 flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle on the host cores on a bounded sample of
the same workload.  Under torchrun every rank runs its own replica (the
quantizer has no cross-rank data dependency; weak scaling) and the timing is
the maximum over ranks.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "quantize+verify GB/s & % HBM peak; residual bits/value learned vs plain"
BOUNDS = ["abs", "rel", "noa"]
EBS = [1e-2, 1e-3, 1e-4, 1e-5]
SHAPE = (512, 512, 512)
WORKLOAD = ("quantize+verify sweep {ABS,REL,NOA} x eb {1e-2,1e-3,1e-4,1e-5} on a float32 "
            "512^3 field (8 random 3-D sinusoids + N(0,0.01)), outlier compaction included")
KERNEL_SOURCES = ["paper_2407_15037_b300/csrc/lcq_quant.cu", "paper_2407_15037_b300/csrc/lcq_device.cuh",
                  "paper_2407_15037_b300/csrc/lcq_pipe.cuh", "paper_2407_15037_b300/csrc/lcq_tile.cuh"]


def kernel_sha():
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


def ncu_traffic(name):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)
    from one ncu capture, as recorded in profiles/traffic.json together with
    the hash of the kernel sources it was taken on; None if absent or if the
    kernel sources changed since the capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)[name]
        return float(rec["bytes_per_launch"]) if rec["kernel_src_sha"] == kernel_sha() else None
    except (OSError, KeyError, TypeError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def step_config(world):
    """The workload of one step (both arms report the same)."""
    return {"workload": WORKLOAD, "n_values": SHAPE[0] * SHAPE[1] * SHAPE[2], "bound_types": BOUNDS,
            "bounds": EBS, "parallelism": "replicas x%d" % world,
            "l2": "inputs larger than L2 (512 MiB per pass vs 126 MB), no flush"}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        if args.impl == "ours":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world, device):
    if world == 1:
        return v
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------ oracle arm --

def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sweep_seconds(xh, threads=1):
    """Time the CPU oracle, as it stands, over the 12-pass sweep of xh:
    quantize_with on one thread, or quantize_parallel (contiguous chunks on
    `threads` host threads; the C code releases the GIL)."""
    import oracle as O
    t0 = time.perf_counter()
    for bound in BOUNDS:
        for eb in EBS:
            c = O.consts(bound, xh.dtype, eb, x=xh)
            if threads == 1:
                O.quantize_with(c, xh)
            else:
                O.quantize_parallel(c, xh, threads=threads)
    return time.perf_counter() - t0


def field_prefix(n, local):
    """The first n values of the benchmark's float32 512^3 field (seed 0):
    generated on the GPU exactly as the timed arm generates it when one is
    visible (then copied to the host), else on the host (same recipe, other
    random draws)."""
    import synth
    if torch.cuda.is_available():
        dev = torch.device("cuda", local)
        x = synth.smooth_field(SHAPE, dtype=torch.float32, seed=0, device=dev)
        xh = x[:n].cpu().numpy()
        del x
        torch.cuda.empty_cache()
        return xh, "the GPU-generated field"
    x = synth.smooth_field(SHAPE, dtype=torch.float32, seed=0, device="cpu")
    return x[:n].numpy().copy(), "the field generated on the host (no GPU visible)"


REF_SAMPLE = 1 << 24


def run_reference(args, world, rank, local):
    if rank != 0:
        return
    cores = host_cores()
    xh, where = field_prefix(REF_SAMPLE, local)
    for _ in range(args.warmup):
        oracle_sweep_seconds(xh, cores)
    t = 0.0
    for _ in range(args.steps):
        t += oracle_sweep_seconds(xh, cores)
    gbs = args.steps * len(BOUNDS) * len(EBS) * xh.nbytes / t / 1e9
    sample = ("first 2^24 values (32 of 512 planes) of %s, float32 512^3 sinusoid field; each step the "
              "12-pass sweep {ABS,REL,NOA} x eb {1e-2,1e-3,1e-4,1e-5} of that sample; oracle over %d host "
              "threads (contiguous chunks)" % (where, cores))
    cfg = step_config(world)
    cfg["timed_sample"] = sample
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- our arm --

def link_bandwidth(h_up, h_down, d_buf, dev, reps=4):
    """Host <-> device copy rates of this machine with the bench's own pinned
    buffers: upload alone, download alone, and both at once on two streams."""
    nb = min(h_up.numel() * h_up.element_size(), h_down.numel() * h_down.element_size(), d_buf.numel() // 2)
    up_src = h_up.view(torch.uint8)[:nb]
    dn_dst = h_down.view(torch.uint8)[:nb]
    d_up, d_dn = d_buf[:nb], d_buf[nb:2 * nb]
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def run(up, down):
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        for _ in range(reps):
            if up:
                with torch.cuda.stream(s1):
                    d_up.copy_(up_src, non_blocking=True)
            if down:
                with torch.cuda.stream(s2):
                    dn_dst.copy_(d_dn, non_blocking=True)
        torch.cuda.synchronize(dev)
        return reps * nb * (int(up) + int(down)) / (time.perf_counter() - t) / 1e9

    run(True, True)
    return {"h2d_GBps": run(True, False), "d2h_GBps": run(False, True), "both_GBps": run(True, True),
            "bytes_per_copy": nb}


def run_lossless(P, x, q, ws, dev, stream, reps=5):
    """The lossless stage after quantization on the float32 512^3 field:
    bins, or the hierarchical-interpolation residuals of the bins, packed into
    bit-planes (lcq_pack).  Compression ratio = input bytes / (packed codes +
    outlier mask + outliers + header); times of encode (residuals + pack) and
    decode (unpack + reconstruct), each checked to give the bins back."""
    from paper_2407_15037_b300 import predictor as PD
    L = P.lcq
    n = x.numel()
    N = SHAPE[0]
    res = {}
    buf = torch.empty(int(L.lib().lcq_pack_bound(n)), dtype=torch.uint8, device=dev)
    pws = torch.empty(int(L.lib().lcq_pack_workspace_size(n)), dtype=torch.uint8, device=dev)

    def timed(fn):
        fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    for bound, eb in (("abs", 1e-3), ("abs", 1e-4), ("rel", 1e-3)):
        P.quantize_into(x, bound, eb, q, ws, stream)
        h = q.read_header()
        side = (n + 31) // 32 * 4 + 4 * h.outlier_count + P.lcq.HEADER_BYTES
        for pred in (False, True):
            key = "%s_%g_%s" % (bound, eb, "interp" if pred else "bins")
            state = {}

            def enc():
                codes = PD.residuals(q.bins, N) if pred else q.bins
                state["size"] = L.pack(codes, buf, pws, stream)[1]

            t_enc = timed(enc)
            size = int(state["size"].item())
            packed = buf[:size]

            def dec():
                codes = L.unpack(packed, n, pws, stream, check=False)
                state["bins"] = PD.reconstruct(codes, N) if pred else codes

            t_dec = timed(dec)
            assert torch.equal(state["bins"], q.bins), key
            total = size + side
            res[key] = {"packed_bytes": size, "total_bytes": total, "ratio": n * 4 / total,
                        "bits_per_value": 8 * total / n, "encode_ms": t_enc, "decode_ms": t_dec,
                        "encode_in_GBps": n * 4 / t_enc / 1e6, "decode_out_GBps": n * 4 / t_dec / 1e6}
    del buf, pws
    return res


def run_ablations(P, x, q, ws, dev, stream, reps=5):
    """The paper's two ablations on the float32 512^3 field: ABS without the
    double-check (Sec. 6, Tables 7-8: time and exact bound violations) and REL
    with the CUDA library's log2/exp2 (Sec. 2.3, Tables 4-6: time, outliers,
    and how many of a sample of its values the host C library's exp2f decodes
    differently).  Each ablation and its protected counterpart run the same
    tile-shape variant."""
    import ctypes
    import ctypes.util
    L = P.lcq
    n = x.numel()

    def timed(fn):
        fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    res = {}
    qa = L.alloc_outputs(n, x.dtype, dev)
    libm = ctypes.CDLL(ctypes.util.find_library("m"))
    libm.exp2f.argtypes = [ctypes.c_float]
    libm.exp2f.restype = ctypes.c_float
    for kind, bound in (("abs_no_check", "abs"), ("rel_library", "rel")):
        v = L.ablation_variant(P.F32, kind)
        keep_v = L.get_variant(0, P.F32, bound)
        L.set_variant(0, P.F32, bound, v)
        for eb in (1e-3, 1e-5):
            t_p = timed(lambda: P.quantize_into(x, bound, eb, q, ws, stream))
            t_a = timed(lambda: L.quantize_ablation_into(x, kind, eb, qa, ws, stream))
            hp, ha = q.read_header(), qa.read_header()
            r = {"variant": v, "protected_ms": t_p, "ablation_ms": t_a,
                 "protected_in_GBps": n * 4 / t_p / 1e6, "ablation_in_GBps": n * 4 / t_a / 1e6,
                 "protected_outliers": int(hp.outlier_count), "ablation_outliers": int(ha.outlier_count)}
            if kind == "abs_no_check":
                r["ablation_bound_violations"] = L.count_abs_violations(x, P.dequantize(qa, ws), eb)
                r["protected_bound_violations"] = L.count_abs_violations(x, P.dequantize(q, ws), eb)
            else:
                m_gpu = L.rel_library_reconstruct(qa)
                idx = torch.nonzero(qa.bins != 0)[:65536, 0]   # accepted values (bin 0 is an outlier or 1.0)
                bins = qa.bins[idx].cpu().numpy()
                mg = m_gpu[idx].cpu().numpy()
                step = np.array([ha.scale_bits], dtype=np.uint64).astype(np.uint32).view(np.float32)[0]
                Lr = (bins >> 1).astype(np.float32) * np.float32(step)
                mc = np.array([libm.exp2f(float(v_)) for v_ in Lr], dtype=np.float32)
                mc = np.where(bins & 1, -mc, mc).astype(np.float32)
                differ = mc.view(np.uint32) != mg.view(np.uint32)
                r["host_exp2f_decode_sample"] = int(bins.size)
                r["host_exp2f_decode_mismatches"] = int(differ.sum())
                r["host_exp2f_max_ulp_diff"] = int(np.abs(mc.view(np.int32).astype(np.int64) -
                                                          mg.view(np.int32).astype(np.int64)).max())
            res["%s_%g" % (kind, eb)] = r
        L.set_variant(0, P.F32, bound, keep_v)
    del qa
    return res


def run_ours(args, world, rank, local):
    import paper_2407_15037_b300 as P
    import synth
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    x = synth.smooth_field(SHAPE, dtype=torch.float32, seed=0, device=dev)
    n = x.numel()
    q = P.alloc_outputs(n, x.dtype, dev)
    ws = P.new_workspace(n, dev)

    abs_events = []  # (start, end) around the consecutive ABS calls of each timed step

    def step(record=False):
        for bound in BOUNDS:
            timed = record and bound == "abs"
            if timed:
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
            for eb in EBS:
                P.quantize_into(x, bound, eb, q, ws, stream)
            if timed:
                b.record(stream)
                abs_events.append((a, b))

    # autotune the tile shape per bound type on this workload (untimed)
    tuning = {}
    for bound in BOUNDS:
        ms = P.lcq.autotune_quantize(x, bound, 1e-3, q, ws, reps=3, stream=stream)
        tuning["quantize_" + bound] = {"chosen": P.lcq.get_variant(0, P.F32, bound),
                                       "ms_per_variant": [round(m, 4) for m in ms]}
    P.quantize_into(x, "abs", 1e-3, q, ws, stream)
    out_t = torch.empty_like(x)
    ms = P.lcq.autotune_dequantize(q, out_t, ws, reps=3, stream=stream)
    tuning["dequantize"] = {"chosen": P.lcq.get_variant(1, P.F32, "abs"),
                            "ms_per_variant": [round(m, 4) for m in ms]}
    del out_t

    # each call: k_quantize, k_compact; NOA calls also k_minmax
    launches_per_step = 2 * len(BOUNDS) * len(EBS) + len(EBS)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize(dev)
    sampler.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(record=True)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    barrier(world)
    ms = e0.elapsed_time(e1)
    ms = max_over_ranks(ms, world, dev)
    bytes_step = len(BOUNDS) * len(EBS) * x.numel() * 4
    value = world * args.steps * bytes_step / (ms / 1e3) / 1e9

    # ---- per-call times: the median of 9 event-timed calls after one untimed
    # call (the paper's convention), CUDA events on the launching stream ----
    per = {}
    for bound in BOUNDS:
        for eb in EBS:
            P.quantize_into(x, bound, eb, q, ws, stream)
            evs = []
            for _ in range(9):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                P.quantize_into(x, bound, eb, q, ws, stream)
                b.record(stream)
                evs.append((a, b))
            torch.cuda.synchronize(dev)
            h = q.read_header()
            t = float(np.median([a.elapsed_time(b) for a, b in evs])) / 1e3
            per["%s_%g" % (bound, eb)] = {"ms": t * 1e3, "outliers": int(h.outlier_count),
                                         "in_GBps": n * 4 / t / 1e9}
    peaks, peak_kind = measured_peaks()
    hbm_peak = float(peaks["hbm_gbs"])
    # dominant kernel: k_quantize<float, ABS> (ABS and NOA calls, 8 of 12 per step); its
    # average launch time over the ABS calls of the timed steps (each ABS call is one launch
    # of it, with its compaction; one event pair brackets the 4 consecutive ABS calls of a
    # step, so that no event sits between two kernels of a call)
    abs_keys = ["abs_%g" % e for e in EBS]
    t_abs = float(np.mean([a.elapsed_time(b) for a, b in abs_events])) / len(EBS) / 1e3
    outl_abs = float(np.mean([per[k]["outliers"] for k in abs_keys]))
    alg_bytes = n * (4 + 4) + (n + 31) // 32 * 4 + 4 * outl_abs  # in + bins + mask + payload
    achieved = alg_bytes / t_abs / 1e9
    traffic = ncu_traffic("k_quantize_f32_abs_512")
    for k, v in per.items():
        v["hbm_GBps"] = (n * 8 + (n + 31) // 32 * 4 + 4 * v["outliers"] +
                         (n * 4 if k.startswith("noa") else 0)) / (v["ms"] / 1e3) / 1e9
        v["pct_hbm_peak"] = 100 * v["hbm_GBps"] / hbm_peak

    # ---- dequantize (device) ----
    out = torch.empty_like(x)
    dstat = torch.zeros(1, dtype=torch.int32, device=dev)
    P.quantize_into(x, "abs", 1e-3, q, ws, stream)
    P.dequantize_into(q, out, ws, dstat, stream)
    evs = []
    for _ in range(9):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        P.dequantize_into(q, out, ws, dstat, stream)
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize(dev)
    t_deq = float(np.median([a.elapsed_time(b) for a, b in evs])) / 1e3

    # ---- other configurations of the same path (timed per call) ----
    extra = {}
    pred_res = None

    def time_calls(xx, bound, eb, reps=10):
        qq = P.alloc_outputs(xx.numel(), xx.dtype, dev)
        ww = P.new_workspace(xx.numel(), dev)
        P.quantize_into(xx, bound, eb, qq, ww, stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            P.quantize_into(xx, bound, eb, qq, ww, stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        t = a.elapsed_time(b) / reps / 1e3
        h = qq.read_header()
        es = xx.element_size()
        alg = xx.numel() * (es + 4) + (xx.numel() + 31) // 32 * 4 + es * h.outlier_count + \
            (xx.numel() * es if bound == "noa" else 0)
        return {"ms": t * 1e3, "in_GBps": xx.numel() * es / t / 1e9, "hbm_GBps": alg / t / 1e9,
                "outliers": int(h.outlier_count)}

    if args.extras:
        # the 1-D sine configuration with planted specials and bin-edge values
        # (2^20 float32, ABS 1e-3): 4 MiB, about 1.3 us of HBM time, so the
        # call is bound by launch latency and has no roofline target
        xc = synth.sine_1d(1 << 20, seed=0, eb=1e-3, device=dev)
        extra["sine_1d_2^20_abs_1e-3"] = time_calls(xc, "abs", 1e-3, reps=50)
        extra["sine_1d_2^20_abs_1e-3"]["note"] = ("launch-bound (4 MiB in, ~1.3 us of HBM time); "
                                                  "mean of 50 back-to-back calls; no roofline target")
        del xc
        extra["ablations"] = run_ablations(P, x, q, ws, dev, stream)
        extra["lossless"] = run_lossless(P, x, q, ws, dev, stream)
        # float64: two roofs, HBM bandwidth and the FP64 multiply rate (probe)
        fp64_rate = P.lcq.fp64_mul_rate(dev)
        extra["fp64_mul_rate_G_per_s"] = fp64_rate / 1e9
        x64 = synth.smooth_field((256, 256, 256), dtype=torch.float64, seed=0, device=dev)
        q64 = P.alloc_outputs(x64.numel(), x64.dtype, dev)
        w64 = P.new_workspace(x64.numel(), dev)
        for bound in BOUNDS:
            P.lcq.autotune_quantize(x64, bound, 1e-3, q64, w64, reps=3, stream=stream)
            for eb in EBS:
                r = time_calls(x64, bound, eb)
                r["variant"] = P.lcq.get_variant(0, P.F64, bound)
                # FP64 operations per value on the common path: the bin's
                # multiplication (ABS, NOA); REL also log2approx's addition
                ops = 2 if bound == "rel" else 1
                r["fp64_ops_per_value"] = ops
                r["fp64_G_per_s"] = ops * x64.numel() / (r["ms"] / 1e3) / 1e9
                r["fp64_frac"] = r["fp64_G_per_s"] * 1e9 / fp64_rate
                r["hbm_frac"] = r["hbm_GBps"] / hbm_peak
                r["nearer_roof"] = "fp64" if r["fp64_frac"] > r["hbm_frac"] else "hbm"
                extra["f64_256_%s_%g" % (bound, eb)] = r
        del q64, w64
        del x64
        # the float32 512^3 field rounded to binary16 / bfloat16
        for fmt, dt in (("f16", torch.float16), ("bf16", torch.bfloat16)):
            xh = synth.smooth_field(SHAPE, dtype=torch.float32, seed=0, device=dev).to(dt)
            qh = P.alloc_outputs(xh.numel(), dt, dev)
            wh = P.new_workspace(xh.numel(), dev)
            code = P.lcq.DTYPE_CODES[dt]
            for bound in BOUNDS:
                P.lcq.autotune_quantize(xh, bound, 1e-3, qh, wh, reps=3, stream=stream)
                key = "%s_512_%s_1e-3" % (fmt, bound)
                extra[key] = time_calls(xh, bound, 1e-3)
                extra[key]["variant"] = P.lcq.get_variant(0, code, bound)
            del qh, wh, xh
        if args.batched:
            extra["batched_4096"] = run_batched(P, synth, dev, stream, args)
        if args.predictor:
            pred_res = run_predictor(P, synth, dev, args)
        xs = synth.rel_stress(1 << 28, seed=0, device=dev)
        for eb in (1e-3, 1e-6):
            extra["rel_stress_2^28_%g" % eb] = time_calls(xs, "rel", eb)
        del xs

    # ---- end to end through the C ABI with host buffers ----
    # The step's 12 quantizations of the host-resident field, each with its
    # own upload and download, through lcq_quantize_host_batch (uploads of one
    # item overlap the downloads of the previous one); for comparison, the
    # same 12 as separate lcq_quantize_host calls.
    e2e = None
    if args.e2e_steps > 0:
        xh = x.cpu().pin_memory()
        cap = n // 16

        def outputs():
            return P.Quantized(torch.empty(n, dtype=torch.int32).pin_memory(),
                               torch.empty((n + 31) // 32, dtype=torch.int32).pin_memory(),
                               torch.empty(cap, dtype=torch.int32).pin_memory(),
                               torch.empty(P.lcq.HEADER_BYTES, dtype=torch.uint8).pin_memory(), n, x.dtype)

        jobs = [(xh, bound, eb, outputs()) for bound in BOUNDS for eb in EBS]
        items = P.lcq.host_items(jobs)
        del q
        stage = torch.empty(P.lcq.host_batch_stage_size(items), dtype=torch.uint8, device=dev)

        def d2h_bytes():
            tot = 0
            for _, _, _, o in jobs:
                hdr = P.Header.from_buffer_copy(o.header.numpy().tobytes())
                tot += n * 4 + (n + 31) // 32 * 4 + P.lcq.HEADER_BYTES + 4 * min(hdr.outlier_count, cap)
            return tot

        def timed(fn, steps):
            fn()
            barrier(world)
            t0 = time.perf_counter()
            for _ in range(steps):
                fn()
            torch.cuda.synchronize(dev)
            return max_over_ranks(time.perf_counter() - t0, world, dev)

        def batch_step():
            st_codes = P.lcq.quantize_host_batch(items, stage, ws, stream, dev)
            assert all(c == 0 for c in st_codes), st_codes

        def single_step():
            for xx, bound, eb, o in jobs:
                P.quantize_host(xx, bound, eb, o, stage, ws, stream, dev)

        te = timed(batch_step, args.e2e_steps)
        d2h = d2h_bytes()
        ts = timed(single_step, args.e2e_steps)
        link = link_bandwidth(xh, jobs[0][3].bins, stage, dev)
        # the step's bytes at the measured concurrent host<->device rate
        t_link = (bytes_step + d2h) / (link["both_GBps"] * 1e9)
        e2e = {"value": world * args.e2e_steps * bytes_step / te / 1e9, "unit": "GB/s",
               "h2d_bytes_per_step": bytes_step, "d2h_bytes_per_step": int(d2h),
               "steps": args.e2e_steps,
               "api": "lcq_quantize_host_batch of the 12 quantizations (pinned host buffers, one output set "
                      "per item)",
               "separate_calls_GBps": world * args.e2e_steps * bytes_step / ts / 1e9,
               "link": link, "link_bound_GBps": bytes_step / t_link / 1e9,
               "frac_of_link_bound": (bytes_step / (te / args.e2e_steps)) / (bytes_step / t_link)}
        del stage, jobs, items

    cpu = None
    if rank == 0 and args.cpu_baseline:
        # the oracle on this machine's host cores, median of 3 runs each: over all
        # cores on the first 2^27 values (half) of the same field, and on one
        # thread on the first 2^25 values
        cores = host_cores()
        xs = x.reshape(-1)[:1 << 27].cpu().numpy()
        t_all = float(np.median([oracle_sweep_seconds(xs, cores) for _ in range(3)]))
        x1 = xs[:1 << 25]
        t_one = float(np.median([oracle_sweep_seconds(x1, 1) for _ in range(3)]))
        cpu = {"value": len(BOUNDS) * len(EBS) * xs.nbytes / t_all / 1e9, "unit": "GB/s", "cores": cores,
               "kind": "oracle",
               "sample": "first 2^27 values (half) of the same 512^3 field, the full 12-pass sweep, oracle "
                         "over %d host threads in contiguous chunks, median of 3 runs (%.2f s each)" % (
                             cores, t_all),
               "nproc": os.cpu_count(),
               "single_thread": {"value": len(BOUNDS) * len(EBS) * x1.nbytes / t_one / 1e9, "unit": "GB/s",
                                 "cores": 1,
                                 "sample": "first 2^25 values of the same field, the 12-pass sweep, oracle "
                                           "single-threaded, median of 3 runs (%.2f s each)" % t_one}}
        del xs, x1

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": step_config(world),
            "pct_hbm_peak_in": 100 * value / world / hbm_peak,
            "roofline": {"bound": "hbm",
                         "kernel": "k_quantize<float,ABS> with its compaction (k_compact): "
                                   "CUDA events bracket the 4 ABS calls of each timed step",
                         "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "peak_source": peak_kind,
                         "alg_bytes_per_launch": alg_bytes, "traffic": traffic,
                         "avg_launch_ms": t_abs * 1e3, "launches_per_call": 2,
                         "launches_timed": len(abs_events) * len(EBS)},
            "clocks": clocks,
            "gpu_launches": launches_per_step * args.steps,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "per_call": per,
            "dequantize_f32_abs_1e-3": {"ms": t_deq * 1e3, "out_GBps": n * 4 / t_deq / 1e9,
                                        "hbm_GBps": n * 8.125 / t_deq / 1e9},
            "other_configs": extra,
            "autotune": tuning,
            "bits_per_value_learned": pred_res["bits_per_value_learned"] if pred_res else None,
            "bits_per_value_interp": pred_res["bits_per_value_interp"] if pred_res else None,
            "predictor": pred_res,
        }
        print(json.dumps(line), flush=True)


def run_batched(P, synth, dev, stream, args):
    """The batched workload: 4096 float32/float64 arrays, lengths log-uniform
    in [4K, 16M], mixed 1-D/2-D/3-D smooth fields, random bound type and bound
    10^U(-5,-2), quantized by one graph-captured replay (header/range pass,
    one persistent quantize launch, per-array offsets, compaction), tile
    shape autotuned on the batch."""
    t0 = time.perf_counter()
    specs = synth.batch_specs(4096, seed=0)
    need = sum(s["n"] * ((8 if s["dtype"] == torch.float64 else 4) * 2 + 4.2) for s in specs)
    free, _ = torch.cuda.mem_get_info(dev)
    scale = 1.0
    if need > 0.8 * free:
        scale = 0.8 * free / need
        specs = synth.batch_specs(4096, seed=0, total_cap=int(sum(s["n"] for s in specs) * scale))
    items = []
    for sp in specs:
        x = synth.smooth_field(sp["shape"], dtype=sp["dtype"], seed=sp["seed"], device=dev)
        items.append((x, sp["bound"], sp["eb"], P.alloc_outputs(x.numel(), x.dtype, dev)))
    torch.cuda.synchronize(dev)
    t_gen = time.perf_counter() - t0
    batch = P.Batch(items, dev, stream)
    ms_var = batch.autotune(reps=2, stream=stream)
    cs = torch.cuda.Stream(dev)  # graphs are captured on a side stream
    cs.wait_stream(stream)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=cs):
        batch.run(stream=cs)
    stream.wait_stream(cs)
    g.replay()
    torch.cuda.synchronize(dev)
    reps = 3
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        g.replay()
    b.record(stream)
    torch.cuda.synchronize(dev)
    t = a.elapsed_time(b) / reps / 1e3
    info = batch.info
    outl = 0
    for _, _, _, q in items[:: max(1, len(items) // 256)]:
        outl += q.read_header().outlier_count
    # a seeded sample of the full batch against single-array calls, bit for
    # bit: header, bins, mask words and outlier payload
    rng = np.random.default_rng(12345)
    pick = sorted(int(i) for i in rng.choice(len(items), 48, replace=False))
    mism = []
    sws = P.new_workspace(max(it[0].numel() for it in items), dev)
    for i in pick:
        xx, bound, eb, qb = items[i]
        ref = P.quantize_into(xx, bound, eb, P.alloc_outputs(xx.numel(), xx.dtype, dev), sws, stream)
        torch.cuda.synchronize(dev)
        cnt = ref.read_header().outlier_count
        same = (bytes(qb.header.cpu().numpy()) == bytes(ref.header.cpu().numpy()) and
                torch.equal(qb.bins, ref.bins) and torch.equal(qb.mask, ref.mask) and
                torch.equal(qb.outliers[:cnt], ref.outliers[:cnt]))
        if not same:
            mism.append(i)
        del ref
    del sws
    res = {"arrays": info.count, "noa_arrays": info.noa_count, "values": int(info.total_values),
           "bytes_in": int(info.total_bytes_in), "ms": t * 1e3,
           "in_GBps": info.total_bytes_in / t / 1e9,
           "hbm_GBps_lower_bound": (2 * info.total_bytes_in + 4.125 * info.total_values) / t / 1e9,
           "scale_vs_full_workload": scale, "generation_s": t_gen, "variant": P.lcq.get_batch_variant(),
           "ms_per_variant": [round(m, 3) for m in ms_var], "launches_per_replay": 4,
           "checked_vs_single_calls": {"arrays": len(pick), "values": int(sum(items[i][0].numel() for i in pick)),
                                       "mismatched": mism, "sample": "48 arrays, numpy seed 12345"}}
    if mism:
        print("batched: arrays %s differ from their single-array calls" % mism, file=sys.stderr, flush=True)
    del items, batch, g
    torch.cuda.empty_cache()
    return res


def run_predictor(P, synth, dev, args):
    """Learned vs interpolation residual entropy: 64 training and 16 test
    float32 256^3 Gaussian random fields with power spectrum k^-3, quantized
    with ABS 1e-3 by the CUDA quantizer; 21 int8 networks trained on the
    device (QAT, Adam) on the training bins; bits/value on the test bins."""
    from paper_2407_15037_b300 import predictor as PD
    N = 256
    t0 = time.perf_counter()

    def field_bins(seed):
        q = P.quantize(synth.grf(N, seed=seed, device=dev), "abs", 1e-3)
        return q

    train = torch.cat([field_bins(s).bins for s in range(args.pred_train_fields)])
    test = [field_bins(1000 + s) for s in range(args.pred_test_fields)]
    torch.cuda.synchronize(dev)
    t_data = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    s_in = PD.choose_s_in(train[:N ** 3].cpu().numpy(), N, rng)
    tr = PD.Trainer(train, N, samples_per_net=args.pred_samples, seed=1, s_in=s_in, s1=9, s2=6, lr=0.5)
    tr.step()
    mse0 = tr.mean_squared_residual()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.pred_steps - 1):
        tr.step()
    b.record()
    torch.cuda.synchronize(dev)
    t_step = a.elapsed_time(b) / max(1, args.pred_steps - 1)
    mse1 = tr.mean_squared_residual()
    params = tr.freeze()
    bi, bl, per = [], [], []
    for q in test:
        r0 = PD.residuals(q.bins, N)
        r1 = PD.residuals(q.bins, N, params)
        x0, d0 = PD.bits_per_value(r0, N, q.mask)
        x1, d1 = PD.bits_per_value(r1, N, q.mask)
        assert torch.equal(PD.reconstruct(r1, N, params), q.bins)
        bi.append(x0)
        bl.append(x1)
        per.append({"interp_pred_bits": d0["pred_bits"], "learned_pred_bits": d1["pred_bits"]})
    # residual kernels' throughput on one test field (bins in, residuals out)
    q = test[0]
    times = {}
    for name, prm in (("interp", None), ("learned", params)):
        PD.residuals(q.bins, N, prm)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            PD.residuals(q.bins, N, prm)
        e1.record()
        torch.cuda.synchronize(dev)
        t = e0.elapsed_time(e1) / 5 / 1e3
        times[name] = {"ms": t * 1e3, "GBps_bins_in_res_out": 8 * N ** 3 / t / 1e9}
    lsq = lsq_reference(train[:4 * N ** 3].cpu().numpy(), q.bins.cpu().numpy(), N)
    return {"workload": "%d train + %d test float32 %d^3 GRF fields, power k^-3, ABS 1e-3" % (
                args.pred_train_fields, args.pred_test_fields, N),
            "bits_per_value_interp": float(np.mean(bi)), "bits_per_value_learned": float(np.mean(bl)),
            "gain_bits_per_value": float(np.mean(bi) - np.mean(bl)), "per_field": per[:4],
            "s_in": [int(v) for v in s_in], "train_steps": args.pred_steps,
            "samples_per_step": int(tr.samples.numel()), "train_ms_per_step": t_step,
            "train_mse_first": mse0, "train_mse_last": mse1, "data_s": t_data, "residual_kernels": times,
            "lsq_linear_reference": lsq}


def lsq_reference(train_bins, test_bins, N, m=40000, seed=0):
    """Sanity reference: a least-squares linear predictor of the residual
    from the 27 raw coarse-stencil deltas (plus a constant), fitted in float64
    on the host per (level, class) from 4 training fields, evaluated on one
    test field; reported as the expected entropy gain 0.5*log2(var ratio),
    weighted by the share of points of each (level, class)."""
    rng = np.random.default_rng(seed)
    F = train_bins.size // N ** 3
    tb = train_bins.reshape(F, N, N, N).astype(np.int64)
    eb = test_bins.reshape(N, N, N).astype(np.int64)
    total, gain = 0.0, 0.0
    for lv, s in enumerate((4, 2, 1), start=1):
        last = ((N - 1) // (2 * s)) * (2 * s)
        c = np.arange(0, N, s)
        for cls in range(1, 8):
            axes = [c[(c // s) % 2 == ((cls >> a) & 1)] for a in range(3)]
            share = np.prod([len(a) for a in axes]) / N ** 3

            def rows(b):
                i, j, k = (rng.choice(a, m) for a in axes)
                acc = np.zeros(m, dtype=np.int64)
                odd = [a for a in range(3) if (cls >> a) & 1]
                for q in range(1 << len(odd)):
                    p = [i.copy(), j.copy(), k.copy()]
                    for bit, a in enumerate(odd):
                        p[a] = np.clip(p[a] + (s if (q >> bit) & 1 else -s), 0, last)
                    acc += b[p[0], p[1], p[2]]
                base = (acc + (1 << (len(odd) - 1))) >> len(odd)
                fi, fj, fk = ((x // (2 * s)) * (2 * s) for x in (i, j, k))
                X = [b[np.clip(fi + 2 * s * di, 0, last), np.clip(fj + 2 * s * dj, 0, last),
                       np.clip(fk + 2 * s * dk, 0, last)] - base
                     for di in (-1, 0, 1) for dj in (-1, 0, 1) for dk in (-1, 0, 1)]
                return np.c_[np.stack(X, 1), np.ones(m)].astype(np.float64), (b[i, j, k] - base).astype(np.float64)
            Xs, Ys = zip(*[rows(tb[f]) for f in range(F)])
            A = np.linalg.lstsq(np.concatenate(Xs), np.concatenate(Ys), rcond=None)[0]
            Xt, Yt = rows(eb)
            v0, v1 = Yt.var(), (Yt - Xt @ A).var()
            gain += share * 0.5 * np.log2(v0 / v1)
            total += share
    return {"expected_gain_bits_per_predicted_value": float(gain / total),
            "expected_gain_bits_per_value": float(gain), "fit": "numpy lstsq float64, 4 fields x 40000 "
            "samples per (level, class), evaluated on a test field"}


def run_profile(args):
    """A short, fixed sequence of calls for ncu captures: three warm-up calls
    and one measured call of the chosen kind on the 512^3 float32 field (or
    the float64 256^3 field, the float32 field rounded to binary16 /
    bfloat16, or the 2^28-value REL stress input)."""
    import paper_2407_15037_b300 as P
    import synth
    dev = torch.device("cuda", 0)
    if args.profile == "pred":
        # the predictor's residual kernels on a 256^3 k^-3 field (ABS 1e-3 bins):
        # interpolation, then the network with seeded int8 weights
        from paper_2407_15037_b300 import predictor as PD
        N = 256
        qp = P.quantize(synth.grf(N, seed=1000, device=dev).reshape(-1), "abs", 1e-3)
        rng = np.random.default_rng(0)
        pp = PD.PredParams()
        w1 = rng.integers(-20, 21, 3 * 7 * 16 * 28)
        for k in range(len(w1)):
            pp.w1[k] = int(w1[k]) if k % 28 != 27 else 0
        for k in range(3 * 7 * 16):
            pp.b1[k] = int(rng.integers(-500, 500))
            pp.w2[k] = int(rng.integers(-20, 21))
        for k in range(21):
            pp.b2[k] = int(rng.integers(-100, 100))
        pp.s_in[0], pp.s_in[1], pp.s_in[2], pp.s1, pp.s2 = 3, 3, 2, 8, 6
        params = PD.params_to_device(pp, dev)
        for prm in (None, params):
            for _ in range(2):
                PD.residuals(qp.bins, N, prm)
        torch.cuda.synchronize()
        print("profile run done pred")
        return
    if args.profile == "compact":
        # two REL 1e-3, two REL 1e-5 and two ABS 1e-5 calls on the float32 512^3 field
        x = synth.smooth_field(SHAPE, dtype=torch.float32, seed=0, device=dev)
        q = P.alloc_outputs(x.numel(), x.dtype, dev)
        ws = P.new_workspace(x.numel(), dev)
        for bound, eb in (("rel", 1e-3),) * 2 + (("rel", 1e-5),) * 2 + (("abs", 1e-5),) * 2:
            P.quantize_into(x, bound, eb, q, ws)
        torch.cuda.synchronize()
        print("profile run done compact")
        return
    shape = (256, 256, 256) if args.profile_dtype == "f64" else SHAPE
    dt = {"f32": torch.float32, "f64": torch.float64, "f16": torch.float16,
          "bf16": torch.bfloat16}[args.profile_dtype]
    if args.profile_input == "stress":
        x = synth.rel_stress(1 << 28, seed=0, device=dev).to(dt)
    elif args.profile_dtype in ("f16", "bf16"):
        x = synth.smooth_field(shape, dtype=torch.float32, seed=0, device=dev).to(dt)
    else:
        x = synth.smooth_field(shape, dtype=dt, seed=0, device=dev)
    q = P.alloc_outputs(x.numel(), x.dtype, dev)
    ws = P.new_workspace(x.numel(), dev)
    out = torch.empty_like(x)
    kind = args.profile
    if kind == "deq":
        P.quantize_into(x, "abs", 1e-3, q, ws)
    for _ in range(4):
        if kind == "deq":
            P.dequantize_into(q, out, ws)
        else:
            P.quantize_into(x, kind, args.profile_eb, q, ws)
    torch.cuda.synchronize()
    print("profile run done", kind, args.profile_dtype)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--profile", choices=["abs", "rel", "noa", "deq", "pred", "compact"], default=None)
    ap.add_argument("--profile-dtype", choices=["f32", "f64", "f16", "bf16"], default="f32")
    ap.add_argument("--profile-input", choices=["smooth", "stress"], default="smooth")
    ap.add_argument("--profile-eb", type=float, default=1e-3)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-extras", dest="extras", action="store_false")
    ap.add_argument("--no-batched", dest="batched", action="store_false")
    ap.add_argument("--no-predictor", dest="predictor", action="store_false")
    ap.add_argument("--pred-train-fields", type=int, default=64)
    ap.add_argument("--pred-test-fields", type=int, default=16)
    ap.add_argument("--pred-steps", type=int, default=2000)
    ap.add_argument("--pred-samples", type=int, default=262144)
    args = ap.parse_args()
    if args.profile:
        run_profile(args)
        return
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
