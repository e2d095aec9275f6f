"""Exhaustive float32 runs of the oracle (Sec. 6: LC was run on all ~4 billion
float32 values at several bounds without a violation).

Every bit pattern is quantized, reconstructed and checked with the exact
verifier.  The default suite runs ABS and NOA over all 2^32 patterns at one
bound and REL over a strided subset; LCQ_EXHAUSTIVE=1 runs all three bound
types over all 2^32 patterns at 1e-2, 1e-3, 1e-4 and 1e-5.
"""
import numpy as np
import pytest

import oracle as O

FULL = 1 << 32
FLT_MAX = float(np.finfo(np.float32).max)


def _full_range_noa(eps):
    # over all float32 patterns the finite min/max are -FLT_MAX and FLT_MAX
    return O.consts("noa", np.float32, eps, rng=(True, -FLT_MAX, FLT_MAX))


def test_abs_all_patterns_1e3():
    c = O.consts("abs", np.float32, 1e-3)
    outl, bad, _ = O.sweep_f32_parallel(c, 0, FULL, 1e-3)
    assert bad == 0
    # at least NaN/Inf/huge values are outliers
    assert outl >= 2 * ((1 << 23) + 1)


def test_noa_all_patterns_1e3():
    c = _full_range_noa(1e-3)
    assert c.all_outliers == 0 and c.R == 2 * FLT_MAX
    outl, bad, _ = O.sweep_f32_parallel(c, 0, FULL, c.eb_abs)
    assert bad == 0


def test_rel_strided_patterns_1e3():
    c = O.consts("rel", np.float32, 1e-3)
    # 1/16 of all patterns: every exponent and sign, strided mantissas
    total_bad = 0
    for start in range(0, FULL, 1 << 28):
        outl, bad, _ = O.sweep_f32_parallel(c, start, 1 << 24, 1e-3)
        total_bad += bad
    assert total_bad == 0


@pytest.mark.slow
@pytest.mark.parametrize("bound", ["abs", "rel", "noa"])
@pytest.mark.parametrize("eps", [1e-2, 1e-3, 1e-4, 1e-5])
def test_all_patterns(bound, eps):
    if bound == "noa":
        c = _full_range_noa(eps)
        ebv = c.eb_abs
    else:
        c = O.consts(bound, np.float32, eps)
        ebv = eps
    outl, bad, inexact = O.sweep_f32_parallel(c, 0, FULL, ebv)
    print("exhaustive", bound, eps, "outliers", outl, "inexact", inexact, "violations", bad)
    assert bad == 0
