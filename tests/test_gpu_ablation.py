"""The ablation kernels on the CUDA path.

Unprotected ABS (Sec. 6, Tables 7-8): bit for bit equal to the oracle's
unprotected quantizer, decoded by the ordinary decoder, and its exact
violation count on the device equal to the oracle's exact verifier.

Library REL (Sec. 2.3, Tables 4-6): every value the device accepted decodes
(with the device library) within the REL bound; the ordinary decoder refuses
the result; decoding the same bins with the host C library gives different
values for some of them, which is the mismatch the paper's approximations
remove."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2407_15037_b300 as P
from paper_2407_15037_b300 import lcq as L
import synth

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _mask_bits(mask, n):
    idx = np.arange(n)
    return ((mask.view(np.uint32)[idx >> 5] >> (idx & 31)) & 1).astype(bool)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("n", [1, 4097, 300001])
def test_unprotected_abs_matches_oracle(dtype, n):
    g = torch.Generator(device=DEV).manual_seed(n)
    x = (torch.randn(n, generator=g, device=DEV, dtype=torch.float64) *
         10.0 ** (torch.rand(n, generator=g, device=DEV, dtype=torch.float64) * 12 - 4)).to(dtype)
    x[::997] = float("nan")
    x[5::1999] = float("inf")
    eb = 1e-3
    q = L.quantize_ablation(x, "abs_no_check", eb)
    h = q.read_header()
    xh = x.cpu().numpy()
    oq = O.quantize_unprotected(xh, eb)
    assert h.status == 0 and h.mode == 0 and h.outlier_count == oq.count
    assert np.array_equal(q.bins.cpu().numpy(), oq.bins)
    assert np.array_equal(q.mask.cpu().numpy().view(np.uint32), oq.mask)
    u = np.uint32 if dtype == torch.float32 else np.uint64
    assert np.array_equal(q.outliers[:oq.count].cpu().numpy().view(u), oq.payload)
    xr = P.dequantize(q)
    assert np.array_equal(xr.cpu().numpy().view(u), O.dequantize(oq).view(u))
    assert L.count_abs_violations(x, xr, eb) == O.verify_abs(xh, xr.cpu().numpy(), eb)


def test_unprotected_abs_breaks_the_bound_where_protected_does_not():
    g = torch.Generator(device=DEV).manual_seed(5)
    x = torch.rand(1 << 20, generator=g, device=DEV) * 1e4 + 1e4  # |x| / eb ~ 1e7
    eb = 1e-3
    qu = L.quantize_ablation(x, "abs_no_check", eb)
    qp = P.quantize(x, "abs", eb)
    bad_u = L.count_abs_violations(x, P.dequantize(qu), eb)
    bad_p = L.count_abs_violations(x, P.dequantize(qp), eb)
    assert bad_u > 0 and bad_p == 0
    assert bad_u == O.verify_abs(x.cpu().numpy(), P.dequantize(qu).cpu().numpy(), eb)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_count_abs_violations_near_the_threshold(dtype):
    rng = np.random.default_rng(9)
    n = 200000
    eb = 1e-3
    npd = np.float32 if dtype == torch.float32 else np.float64
    x = rng.uniform(-10, 10, n).astype(npd)
    # differences within a few units in the last place of eb, both signs
    d = eb * (1.0 + rng.integers(-4, 5, n) * np.finfo(npd).eps) * rng.choice([-1.0, 1.0], n)
    xr = (x.astype(np.float64) + d).astype(npd)
    xr[:100] = x[:100]
    xr[100:110] = np.nan
    x[110:120] = np.nan
    xr[110:120] = x[110:120]
    got = L.count_abs_violations(torch.from_numpy(x).to(DEV), torch.from_numpy(xr).to(DEV), eb)
    assert got == O.verify_abs(x, xr, eb)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_rel_library_variant(dtype):
    x = synth.rel_stress(1 << 20, seed=3, device=DEV).to(dtype)
    eb = 1e-3
    q = L.quantize_ablation(x, "rel_library", eb)
    h = q.read_header()
    assert h.status == 0 and h.mode == 2 and h.bound_type == P.REL
    npd, u = (np.float32, np.uint32) if dtype == torch.float32 else (np.float64, np.uint64)
    c = O.consts("rel", npd, eb)
    assert h.scale_bits == int(np.array([c.step]).astype(npd).view(u)[0])
    # the ordinary decoder refuses a library-variant result
    with pytest.raises(P.LcqError):
        P.dequantize(q)
    m_gpu = L.rel_library_reconstruct(q).cpu().numpy()
    xh = x.cpu().numpy()
    out = _mask_bits(q.mask.cpu().numpy(), x.numel())
    # zeros, denormals, NaN/Inf are outliers as in the approximation variant
    specials = ~np.isfinite(xh) | (np.abs(xh) < np.finfo(xh.dtype).tiny)
    assert np.all(out[specials])
    keep = ~out
    assert O.verify_rel(xh[keep], m_gpu[keep], eb) == 0
    # the same bins decoded with the host C library
    m_cpu = O.rel_library_recon(xh.dtype, c.step, q.bins.cpu().numpy(), q.mask.cpu().numpy().view(np.uint32))
    differ = int(np.sum(m_cpu[keep].view(u) != m_gpu[keep].view(u)))
    bad_cpu = O.verify_rel(xh[keep], m_cpu[keep], eb)
    print("rel_library %s: outliers %d of %d, host-decode mismatches %d, host-decode violations %d"
          % (dtype, int(out.sum()), x.numel(), differ, bad_cpu))
    assert bad_cpu <= differ


def test_rel_library_reconstruct_refuses_other_headers():
    x = synth.smooth_field((5000,), seed=1, device=DEV)
    q = P.quantize(x, "rel", 1e-3)
    with pytest.raises(P.LcqError):
        L.rel_library_reconstruct(q)
