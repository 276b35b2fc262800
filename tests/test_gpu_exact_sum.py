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


@pytest.mark.parametrize("as_float", [False, True])
def test_matches_exact_rational_sum(as_float):
    rng = np.random.default_rng(3)
    for n, span in ((1, 10), (37, 4), (5000, 40), (100000, 58)):
        t = rng.standard_normal(n) * np.exp2(rng.integers(-span, span + 1, n).astype(float))
        if as_float:
            t = t.astype(np.float32).astype(np.float64)
        got = pimc.debug_fix_sum(t, as_float=as_float)
        ref = exact(t)
        assert abs(got - ref) <= math.ulp(ref), (n, got, ref)
        perm = rng.permutation(n)
        assert pimc.debug_fix_sum(t[perm], as_float=as_float) == got


def test_cancellation_is_exact():
    # FP64 summation in this order loses the 1.0 entirely; the exact sum keeps it
    t = np.array([2.0 ** 60, 1.0, -(2.0 ** 60)] * 1000)
    assert pimc.debug_fix_sum(t) == 1000.0
    assert pimc.debug_fix_sum([2.0 ** -70, -(2.0 ** -70), 2.0 ** -65]) == 0.0  # below 2^-64: truncated


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
