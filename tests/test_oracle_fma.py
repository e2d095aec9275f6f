"""The no-FMA build flags are load-bearing (Sec. 2.3 / 3.2): the same oracle
source compiled with FMA contraction allowed (-ffp-contract=fast -mfma) gives
different ABS bins, and some of its accepted values break the bound once
decoded by a decoder that rounds the product (as the GPU decoder and the
normal build do).  The normal build, used everywhere else, gives none."""
import ctypes
import subprocess

import numpy as np
import pytest

import oracle as O
from oracle import build as B


def _cpu_has_fma():
    try:
        return " fma " in " " + open("/proc/cpuinfo").read().replace("\n", " ") + " "
    except OSError:
        return False


@pytest.mark.skipif(not _cpu_has_fma(), reason="host CPU without FMA")
def test_fma_contraction_changes_abs_results(tmp_path):
    flags = [f for f in B.CFLAGS if f not in ("-ffp-contract=off", "-mno-fma")] + ["-ffp-contract=fast", "-mfma"]
    so = tmp_path / "liblcq_oracle_fma.so"
    subprocess.run(["gcc", *flags, "-o", str(so), B.SRC, "-lquadmath", "-lm"], check=True)
    L = ctypes.CDLL(str(so))
    L.lcqo_quantize.argtypes = [ctypes.POINTER(O.Consts), ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64]
    L.lcqo_quantize.restype = ctypes.c_uint64
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(1 << 20) * 10.0 ** rng.uniform(-3, 3, 1 << 20)).astype(np.float32)
    eb = 1e-3
    c = O.consts("abs", np.float32, eb)
    ref = O.quantize_with(c, x)
    n = x.size
    bins = np.empty(n, np.int32)
    mask = np.empty((n + 31) // 32, np.uint32)
    pay = np.empty(n, np.uint32)
    cnt = int(L.lcqo_quantize(ctypes.byref(c), x.ctypes.data, n, bins.ctypes.data, mask.ctypes.data,
                              pay.ctypes.data, n))
    assert np.sum(bins != ref.bins) > 0                      # the flag changes the result
    fused = O.Quantized(bins, mask, pay[:cnt], cnt, c)
    assert O.verify_abs(x, O.dequantize(fused), eb) > 0      # and breaks the guarantee across builds
    assert O.verify_abs(x, O.dequantize(ref), eb) == 0       # the normal build keeps it
