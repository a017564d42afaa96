"""The precision study's CPU emulation (tests/study_emulation.py) rounds each
fused multiply-add once: checked against exact rational arithmetic on random
and constructed tie cases (no GPU)."""
from fractions import Fraction

import numpy as np
import pytest

import study_emulation as S


def exact_rn(v, dtype):
    """Round the rational v to the nearest dtype value, ties to even."""
    f = float(v)  # nearest FP64
    lo = np.array([f]).astype(dtype)[0]
    cands = {float(lo), float(np.nextafter(lo, dtype(np.inf))), float(np.nextafter(lo, dtype(-np.inf)))}
    best = min(cands, key=lambda c: (abs(Fraction(c) - v),
                                     int(np.array([c]).astype(dtype).view(np.uint16 if dtype == np.float16
                                                                              else np.uint32)[0]) & 1))
    return best


@pytest.mark.parametrize("dtype", [np.float16, np.float32])
def test_fma_single_rounding(dtype):
    rng = np.random.default_rng(11)
    a = S.rnd(rng.uniform(-4, 4, 4000), dtype)
    b = S.rnd(rng.uniform(-4, 4, 4000), dtype)
    c = S.rnd(rng.uniform(-8, 8, 4000) * 10.0 ** rng.integers(-6, 2, 4000), dtype)
    got = S.fma(a, b, c, dtype)
    for k in range(a.size):
        want = exact_rn(Fraction(a[k]) * Fraction(b[k]) + Fraction(c[k]), dtype)
        assert got[k] == want, (a[k], b[k], c[k])


def test_fma_tie_with_tiny_addend():
    """a*a exactly halfway between two FP32 values plus an addend far below
    FP64's last bit: a plain FP64 sum would round to the tie and then to even;
    the single rounding goes up."""
    a = np.array([float(4097 * 2.0 ** -12)])       # 4097^2 = 2^24 + 2^13 + 1: 25 bits, an FP32 tie
    p = Fraction(a[0]) ** 2
    c = np.array([2.0 ** -80])
    got = S.fma(a, a, c, np.float32)[0]
    assert got == exact_rn(p + Fraction(c[0]), np.float32)
    assert got > float(np.float32(float(p)))
