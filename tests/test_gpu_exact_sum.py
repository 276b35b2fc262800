"""The exact sum behind every parameter-move decision (42-bit integer chunks
of 2^-64), pinned against exact rational arithmetic: each term truncated
toward zero to a multiple of 2^-64, summed exactly, rounded to FP64 -- the
device result is within one unit in the last place of that value (it rounds
twice) and is the same in every term order."""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_1103_4887_gb300 import pimc

pytestmark = pytest.mark.gpu


def exact(terms):
    s = sum(int(Fraction(float(t)) * (1 << 64)) for t in terms)  # int() truncates toward zero
    return float(Fraction(s, 1 << 64))


@pytest.mark.parametrize("mode", ["fp64", "fp32", "fp32_acc128"])
def test_matches_exact_rational_sum(mode):
    """Also the 128-bit per-thread path of FP32 terms: below 2^36 a term is
    shifted into one 128-bit integer, above it goes through the chunks; both
    sides of that cut, subnormal and sub-2^-64 terms are in the mix."""
    as_float, acc128 = mode != "fp64", mode == "fp32_acc128"
    rng = np.random.default_rng(3)
    for n, span in ((1, 10), (37, 4), (5000, 40), (100000, 58)):
        t = rng.standard_normal(n) * np.exp2(rng.integers(-span, span + 1, n).astype(float))
        if as_float:
            t = t.astype(np.float32).astype(np.float64)
            if n > 1:
                t[:4] = [2.0 ** 36, -(2.0 ** 36) + 2.0 ** 13, 2.0 ** -140, -(2.0 ** -70)]
        got = pimc.debug_fix_sum(t, as_float=as_float, acc128=acc128)
        ref = exact(t)
        assert abs(got - ref) <= math.ulp(ref), (n, got, ref)
        perm = rng.permutation(n)
        assert pimc.debug_fix_sum(t[perm], as_float=as_float, acc128=acc128) == got
        if as_float:  # the two FP32 paths give the same bits
            assert pimc.debug_fix_sum(t, as_float=True, acc128=not acc128) == got


def test_cancellation_is_exact():
    # FP64 summation in this order loses the 1.0 entirely; the exact sum keeps it
    t = np.array([2.0 ** 60, 1.0, -(2.0 ** 60)] * 1000)
    assert pimc.debug_fix_sum(t) == 1000.0
    assert pimc.debug_fix_sum([2.0 ** -70, -(2.0 ** -70), 2.0 ** -65]) == 0.0  # below 2^-64: truncated


@pytest.mark.parametrize("acc128", [False, True])
def test_special_values_fp32(acc128):
    inf, nan = float("inf"), float("nan")
    f = lambda t: pimc.debug_fix_sum(t, as_float=True, acc128=acc128)
    assert f([1.0, inf]) == inf and f([1.0, -inf]) == -inf
    assert math.isnan(f([inf, -inf])) and math.isnan(f([0.5, nan]))
    assert f([2.0 ** 62, -1.0]) == inf
    big = np.full(1 << 20, -(2.0 ** 35))                      # the 128-bit path at its cut, 2^20 times
    assert f(big) == -(2.0 ** 55)


def test_special_values():
    inf, nan = float("inf"), float("nan")
    assert pimc.debug_fix_sum([1.0, inf]) == inf
    assert pimc.debug_fix_sum([1.0, -inf]) == -inf
    assert math.isnan(pimc.debug_fix_sum([inf, -inf]))
    assert math.isnan(pimc.debug_fix_sum([0.5, nan]))
    assert pimc.debug_fix_sum([2.0 ** 62, -1.0]) == inf       # magnitude >= 2^62 counts as infinite
    assert pimc.debug_fix_sum([-(2.0 ** 63)]) == -inf
    assert pimc.debug_fix_sum([]) == 0.0
    big = np.full(1 << 20, 2.0 ** 61 - 2.0 ** 9)               # the largest sum the chunks hold
    assert pimc.debug_fix_sum(big) == exact(big[:1]) * (1 << 20)
    with pytest.raises(pimc.PimcError):
        pimc.debug_fix_sum(np.zeros((1 << 20) + 1))
