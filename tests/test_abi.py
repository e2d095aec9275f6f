"""The C-ABI library loads without a GPU and exports every function that
include/*.h declares; the binding's struct mirrors match the header."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

import paper_2407_15037_b300 as P
from paper_2407_15037_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(lcq_\w+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    B.build()
    return P.lib()


def test_library_exports_every_declared_function(lib):
    declared = _declared_functions()
    assert declared, "no declarations found"
    out = subprocess.run(["nm", "-D", "--defined-only", P.lcq.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = sorted(declared - exported)
    assert not missing, missing
    for name in declared:
        assert hasattr(lib, name)


def test_binding_covers_the_declarations():
    from paper_2407_15037_b300 import predictor as PD
    bound = set(P.lcq.SIGNATURES) | set(PD.SIGNATURES)
    missing = sorted(_declared_functions() - bound)
    assert not missing, missing


def test_header_struct_size_matches_c(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include "lcq.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(lcq_header),'
                   ' offsetof(lcq_header, outlier_count), offsetof(lcq_header, status),'
                   ' sizeof(lcq_batch_item), sizeof(lcq_batch_info), offsetof(lcq_batch_item, d_hdr));'
                   'printf("%zu %zu %zu\\n", sizeof(lcq_pred_params), sizeof(lcq_host_item),'
                   ' offsetof(lcq_host_item, status));'
                   'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-I", "/usr/local/cuda/include",
                    str(src), "-o", str(exe)], check=True)
    size, off_cnt, off_st, bi, binfo, off_hdr, pp, hi, off_hs = map(int, subprocess.run(
        [str(exe)], capture_output=True, text=True, check=True).stdout.split())
    from paper_2407_15037_b300 import predictor as PD
    assert pp == PD.PARAMS_BYTES
    assert hi == ctypes.sizeof(P.lcq.HostItem) and off_hs == P.lcq.HostItem.status.offset
    H = P.Header
    assert size == ctypes.sizeof(H)
    assert off_cnt == H.outlier_count.offset and off_st == H.status.offset
    assert bi == ctypes.sizeof(P.BatchItem) and binfo == ctypes.sizeof(P.BatchInfo)
    assert off_hdr == P.BatchItem.d_hdr.offset


def test_host_side_argument_errors_need_no_gpu(lib):
    # invalid enums and bounds are rejected before anything touches a device
    ws = (ctypes.c_uint8 * 4096)()
    hdr = (ctypes.c_uint8 * 128)()
    p = ctypes.c_void_p(ctypes.addressof(ws) + (-ctypes.addressof(ws)) % 16)
    h = ctypes.c_void_p(ctypes.addressof(hdr) + (-ctypes.addressof(hdr)) % 16)
    assert lib.lcq_quantize(7, 0, 1e-3, None, 0, None, None, None, 0, h, p, 4000, None) == 1
    assert lib.lcq_quantize(0, 9, 1e-3, None, 0, None, None, None, 0, h, p, 4000, None) == 1
    assert lib.lcq_quantize(0, 0, -1.0, None, 0, None, None, None, 0, h, p, 4000, None) == 2
    assert lib.lcq_quantize(0, 0, float("nan"), None, 0, None, None, None, 0, h, p, 4000, None) == 2
    assert lib.lcq_status_string(4) == b"outlier scan wait timed out"
    # a caller-given NOA range: has_finite 0/1, finite, ordered, float values for float32
    nr = lambda dt, has, lo, hi: lib.lcq_quantize_noa_range(dt, 1e-3, has, lo, hi, None, 0, None, None, None, 0,
                                                            h, p, 4000, None)
    assert nr(0, 2, 0.0, 1.0) == 1
    assert nr(0, 1, 1.0, 0.0) == 1
    assert nr(0, 1, float("-inf"), 0.0) == 1
    assert nr(0, 1, 0.0, float("nan")) == 1
    assert nr(0, 1, 0.0, 0.1) == 1          # 0.1 is not a float32 value
    assert lib.lcq_quantize_noa_range(0, -1.0, 1, 0.0, 1.0, None, 0, None, None, None, 0, h, p, 4000, None) == 2
    assert lib.lcq_finite_range(7, None, 0, p, p, 4000, None) == 1
    # 16-bit formats: the range values must be values of the format
    assert nr(2, 1, 0.0, 0.1) == 1               # not a binary16 value
    assert nr(2, 1, 0.0, 65520.0) == 1           # beyond binary16's largest value
    assert nr(3, 1, 0.0, 1.0 + 2.0 ** -10) == 1  # not a bfloat16 value (7 fraction bits)
    assert nr(4, 1, 0.0, 1.0) == 1               # no such data type
    assert lib.lcq_finite_range(0, None, 0, None, p, 4000, None) == 1
    assert lib.lcq_finite_range(0, None, 0, ctypes.c_void_p(p.value + 4), p, 4000, None) == 1
    assert lib.lcq_workspace_size(0, 0, 1 << 31) > lib.lcq_workspace_size(0, 0, 1 << 20)


def test_workspace_size_and_allocation_free_limit(lib):
    """The single-array workspace is the head (256 B), the range partials
    (1184 blocks x 16 B), the group counts of 64 scan tiles at a fixed place
    (8 KB: every chunk of up to 2^31 values has at most 2^17 tiles of 16384
    values), and one uint32 count per 16384-value tile of the largest chunk,
    each region rounded up to 256 B.  Float32 REL adds the outlier staging
    table (one uint64 per ring stage: at most 8 stages per tile) and a
    staging area for a quarter of the largest chunk's values.  Every n below
    2^40 fits the 1 MiB scratch of the allocation-free entry point, which
    does not stage."""
    def up256(b):
        return (b + 255) // 256 * 256

    for n in (0, 1, 16384, 16385, 1 << 20, 134217728, (1 << 31) - 1, 1 << 31, (1 << 31) + 1, 1 << 36):
        per_chunk = min(n, 1 << 31)
        tiles = (per_chunk + 16383) // 16384
        want = 256 + 1184 * 16 + 8192 + up256(4 * tiles)
        staged = want + up256(8 * 8 * tiles) + up256(4 * ((per_chunk + 3) // 4))
        for dtype in (0, 1, 2, 3):
            for bound in (0, 1, 2):
                got = lib.lcq_workspace_size(dtype, bound, n)
                assert got == (staged if (dtype, bound) == (0, 1) else want)
    assert lib.lcq_noalloc_max_values() == (1 << 40) - 1


def test_default_workspace_fits_every_bound(lib):
    """new_workspace without a bound is sized for every bound type of the
    data type, so a float32 REL call on it stages its outliers; with a bound
    it is exactly that bound's size (no device needed: a host tensor)."""
    n = (1 << 20) + 3
    for code in (P.lcq.F32, P.lcq.F64, P.lcq.F16, P.lcq.BF16):
        sizes = [P.workspace_size(code, b, n) for b in ("abs", "rel", "noa")]
        assert P.new_workspace(n, "cpu", code).numel() == max(sizes)
        assert P.new_workspace(n, "cpu", code, "abs").numel() == sizes[0]
    assert P.new_workspace(n, "cpu").numel() == P.workspace_size(P.lcq.F32, "rel", n)
