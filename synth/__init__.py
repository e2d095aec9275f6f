"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the quantizers.  It only builds input
arrays; the CUDA path and the oracle both consume what it returns, and every
array is generated once and copied to whichever side needs it, so both sides
always see identical bits.

The paper measures on SDRBench files (Table 2: smooth 1-D/2-D/3-D float32
fields such as climate, cosmology and weather data, 100^3..512^3 values) and on
generated sets with +/-Inf, NaN and denormals (Sec. 5).  Those files are not
available here; the generators below stand in for them:

  sine_1d      1-D float32, sin(0.001 i) * 100 + N(0, 0.1), with 0.1% of the
               entries replaced by NaNs (quiet, signalling, with payloads),
               +/-Inf, denormals and values placed on and within one ulp of
               ABS bin edges.
  smooth_field sum of 8 random 3-D sinusoids plus N(0, 0.01) noise (any shape
               of 1 to 3 dimensions, float32 or float64).
  rel_stress   log-uniform magnitudes over [1e-30, 1e30], random sign, 10%
               exact zeros, 1% denormals, 0.1% NaN/Inf.
  grf          Gaussian random field with power spectrum |k|^-3, normalised to
               mean 0 and standard deviation 1.
  batch_specs  descriptions of a batch of fields with log-uniform lengths,
               mixed dtype, dimensionality, bound type and bound.
"""
import math

import numpy as np
import torch


def _gen(seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def sine_1d(n=1 << 20, seed=0, eb=1e-3, special_frac=1e-3, device="cpu"):
    """Config of the 1-D ABS test: a sine wave plus noise with planted
    special values and bin-edge values for bound eb."""
    g = _gen(seed, device)
    i = torch.arange(n, device=device, dtype=torch.float64)
    x = (torch.sin(0.001 * i) * 100.0).to(torch.float32)
    x = x + torch.randn(n, generator=g, device=device, dtype=torch.float32) * 0.1
    m = int(round(special_frac * n))
    if m == 0:
        return x
    idx = torch.randperm(n, generator=g, device=device)[:m]
    kinds = torch.arange(m, device=device) % 8
    bits = x.view(torch.int32).clone()
    # 0: quiet NaN, 1: signalling NaN with payload, 2: negative NaN with payload
    r = torch.randint(1, 1 << 22, (m,), generator=g, device=device, dtype=torch.int32)
    vals = torch.zeros(m, dtype=torch.int32, device=device)
    vals = torch.where(kinds == 0, torch.full_like(vals, 0x7FC00000), vals)
    vals = torch.where(kinds == 1, 0x7F800000 | r, vals)
    vals = torch.where(kinds == 2, (0xFFC00000 - (1 << 32)) | r, vals)
    vals = torch.where(kinds == 3, torch.full_like(vals, 0x7F800000), vals)            # +Inf
    vals = torch.where(kinds == 4, torch.full_like(vals, 0xFF800000 - (1 << 32)), vals)  # -Inf
    sign = torch.randint(0, 2, (m,), generator=g, device=device, dtype=torch.int32)
    den = torch.randint(1, 1 << 23, (m,), generator=g, device=device, dtype=torch.int32)
    vals = torch.where(kinds == 5, den | (sign << 31), vals)                            # denormals
    # 6, 7: values on a bin edge (k + 1/2) * 2 eb near the original value,
    # then moved by -1, 0 or +1 ulp.
    xo = x[idx].to(torch.float64)
    k = torch.floor(xo / (2.0 * eb))
    edge = ((k + 0.5) * (2.0 * eb)).to(torch.float32).view(torch.int32)
    shift = torch.randint(-1, 2, (m,), generator=g, device=device, dtype=torch.int32)
    vals = torch.where(kinds >= 6, edge + shift, vals)
    bits[idx] = vals
    return bits.view(torch.float32)


def smooth_field(shape, dtype=torch.float32, seed=0, noise=0.01, device="cpu", terms=8):
    """Sum of `terms` random sinusoids over an integer grid of `shape`
    (1 to 3 dims) plus N(0, noise): amplitudes U[0.5, 2], integer wave
    numbers U{0..8} per axis (not all zero), phases U[0, 2 pi)."""
    shape = tuple(int(s) for s in shape)
    g = _gen(seed, device)
    nd = len(shape)
    acc = torch.zeros(shape, dtype=torch.float64, device=device)
    for _ in range(terms):
        A = 0.5 + 1.5 * torch.rand((), generator=g, device=device, dtype=torch.float64)
        while True:
            w = torch.randint(0, 9, (nd,), generator=g, device=device)
            if int(w.abs().sum()) > 0:
                break
        phi = 2 * math.pi * torch.rand((), generator=g, device=device, dtype=torch.float64)
        ph = phi.clone()
        for ax in range(nd):
            coord = torch.arange(shape[ax], device=device, dtype=torch.float64)
            view = [1] * nd
            view[ax] = shape[ax]
            ph = ph + (2 * math.pi * w[ax].to(torch.float64) / shape[ax] * coord).view(view)
        acc += A * torch.sin(ph)
    x = acc.to(dtype)
    x += (torch.randn(shape, generator=g, device=device, dtype=torch.float64) * noise).to(dtype)
    return x.reshape(-1)


def rel_stress(n=1 << 28, seed=0, device="cpu"):
    """Log-uniform magnitudes 10^U(-30, 30), random sign, then 10% set to
    +/-0, 1% to random denormals and 0.1% to NaN/+Inf/-Inf on disjoint index
    sets."""
    g = _gen(seed, device)
    e = torch.rand(n, generator=g, device=device, dtype=torch.float64) * 60.0 - 30.0
    x = torch.pow(10.0, e).to(torch.float32)
    neg = torch.rand(n, generator=g, device=device) < 0.5
    x = torch.where(neg, -x, x)
    bits = x.view(torch.int32)
    perm = torch.randperm(n, generator=g, device=device)
    nz, nd, ns = n // 10, n // 100, n // 1000
    iz = perm[:nz]
    idn = perm[nz:nz + nd]
    isp = perm[nz + nd:nz + nd + ns]
    sz = torch.randint(0, 2, (nz,), generator=g, device=device, dtype=torch.int32)
    bits[iz] = sz << 31
    sd = torch.randint(0, 2, (nd,), generator=g, device=device, dtype=torch.int32)
    md = torch.randint(1, 1 << 23, (nd,), generator=g, device=device, dtype=torch.int32)
    bits[idn] = md | (sd << 31)
    kind = torch.arange(ns, device=device) % 3
    sp = torch.where(kind == 0, torch.full((ns,), 0x7FC00000, dtype=torch.int32, device=device),
                     torch.where(kind == 1,
                                 torch.full((ns,), 0x7F800000, dtype=torch.int32, device=device),
                                 torch.full((ns,), 0xFF800000 - (1 << 32), dtype=torch.int32,
                                            device=device)))
    bits[isp] = sp
    return bits.view(torch.float32)


def grf(N=256, seed=0, device="cpu", slope=-3.0):
    """Gaussian random field on an N^3 grid with power spectrum |k|^slope
    (k in integer grid units, P(0) = 0), normalised to mean 0, std 1; float32."""
    g = _gen(seed, device)
    w = torch.randn((N, N, N), generator=g, device=device, dtype=torch.float64)
    W = torch.fft.rfftn(w)
    kx = torch.fft.fftfreq(N, d=1.0 / N, device=device, dtype=torch.float64)
    kz = torch.fft.rfftfreq(N, d=1.0 / N, device=device, dtype=torch.float64)
    k2 = kx.view(-1, 1, 1) ** 2 + kx.view(1, -1, 1) ** 2 + kz.view(1, 1, -1) ** 2
    amp = torch.where(k2 > 0, k2.clamp_min(1e-30) ** (slope / 4.0), torch.zeros_like(k2))
    f = torch.fft.irfftn(W * amp, s=(N, N, N))
    f = (f - f.mean()) / f.std()
    return f.to(torch.float32).reshape(-1)


def _near_cubic(n, nd, rng):
    """A factorisation of n into nd near-equal factors (the last absorbs the rest)."""
    if nd == 1:
        return (n,)
    side = max(1, int(round(n ** (1.0 / nd))))
    if nd == 2:
        a = side
        return (a, max(1, n // a))
    a = side
    b = side
    return (a, b, max(1, n // (a * b)))


def batch_specs(count=4096, seed=0, lo=4096, hi=1 << 24, total_cap=None):
    """Descriptions of a batch of fields: length log-uniform in [lo, hi],
    dtype float32/float64 with p = 1/2, 1-D/2-D/3-D shape with a near-cubic
    factorisation, bound type uniform over abs/rel/noa, bound 10^U(-5, -2).

    Returns a list of dicts {shape, n, dtype, bound, eb, seed}.  total_cap,
    if given, scales the lengths down so that their sum stays below it."""
    rng = np.random.default_rng(seed)
    lens = np.round(np.exp(rng.uniform(math.log(lo), math.log(hi), count))).astype(np.int64)
    if total_cap is not None and lens.sum() > total_cap:
        lens = np.maximum(32, (lens * (total_cap / lens.sum())).astype(np.int64))
    specs = []
    for a in range(count):
        nd = int(rng.integers(1, 4))
        shape = _near_cubic(int(lens[a]), nd, rng)
        n = int(np.prod(shape))
        specs.append(dict(
            shape=shape, n=n,
            dtype=torch.float32 if rng.random() < 0.5 else torch.float64,
            bound=("abs", "rel", "noa")[int(rng.integers(0, 3))],
            eb=float(10.0 ** rng.uniform(-5.0, -2.0)),
            seed=int(seed * 100003 + a),
        ))
    return specs
