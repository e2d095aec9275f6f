"""Cases whose outcome the paper fixes (tests/golden/paper_sec2_special_cases.txt, each
group with its section): NaN and INF under ABS and REL, denormals under ABS and REL, and
bins at and beyond the int32 range.  The oracle is checked against the fixture on the CPU;
the CUDA path is checked against the same fixture on the GPU."""
import os

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
FIXTURE = os.path.join(HERE, "golden", "paper_sec2_special_cases.txt")
NP = {"f32": (np.float32, np.uint32), "f64": (np.float64, np.uint64)}


def _rows():
    rows = []
    with open(FIXTURE) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            dt, bound, eb, bits, outl, b = line.split()
            eb = float.fromhex(eb) if eb.startswith("0x") else float(eb)
            rows.append((dt, bound, eb, int(bits, 16), int(outl), None if b == "-" else int(b)))
    return rows


ROWS = _rows()


def _value(dt, bits):
    f, u = NP[dt]
    return np.array([bits], dtype=u).view(f)


def test_fixture_is_complete():
    assert len(ROWS) == 25
    assert {r[0] for r in ROWS} == {"f32", "f64"} and {r[1] for r in ROWS} == {"abs", "rel"}


@pytest.mark.parametrize("row", ROWS, ids=lambda r: "%s-%s-%g-%x" % r[:4])
def test_oracle_matches_fixture(row):
    dt, bound, eb, bits, outl, b = row
    x = _value(dt, bits)
    q = O.quantize(x, bound, eb)
    assert int(q.mask[0] & 1) == outl
    assert q.count == outl
    if outl:
        assert q.bins[0] == 0
        assert q.payload.view(NP[dt][1])[0] == bits  # kept bit for bit
    else:
        assert q.bins[0] == b


@pytest.mark.gpu
@pytest.mark.parametrize("row", ROWS, ids=lambda r: "%s-%s-%g-%x" % r[:4])
def test_cuda_path_matches_fixture(row):
    import torch
    import paper_2407_15037_b300 as P
    dt, bound, eb, bits, outl, b = row
    x = torch.from_numpy(_value(dt, bits).copy()).to("cuda")
    q = P.quantize(x, bound, eb)
    h = q.read_header()
    assert h.status == 0 and h.outlier_count == outl
    assert int(q.mask.cpu().numpy().view(np.uint32)[0] & 1) == outl
    assert int(q.bins.cpu().numpy()[0]) == (0 if outl else b)
    xr = P.dequantize(q).cpu().numpy().view(NP[dt][1])[0]
    if outl:
        assert xr == bits
