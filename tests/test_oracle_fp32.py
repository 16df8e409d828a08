"""Pins of the oracle's binary32 decision arithmetic against exact rational rounding."""
from fractions import Fraction

import numpy as np

from oracle.fp32 import fma32


def round_to_f32(x: Fraction) -> float:
    """Exact round-to-nearest-even of a rational to binary32 (normal range)."""
    if x == 0:
        return 0.0
    sign = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    ulp = Fraction(2) ** (e - 23)
    m = a / ulp
    fl = m.numerator // m.denominator
    rem = m - fl
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and fl % 2 == 1):
        fl += 1
    return sign * float(fl * ulp)


def _check(a, b, c):
    got = fma32(np.float32(a), np.float32(b), np.float32(c))
    ex = Fraction(float(np.float32(a))) * Fraction(float(np.float32(b))) + Fraction(float(np.float32(c)))
    want = np.float32(round_to_f32(ex))
    assert got == want, (a, b, c, got, want)


def test_fma32_random_matches_exact_rounding():
    rng = np.random.default_rng(1)
    for _ in range(3000):
        a, b, c = rng.standard_normal(3) * np.exp(rng.uniform(-8, 8, 3))
        _check(a, b, c)


def test_fma32_near_cancellation_and_halfway_cases():
    rng = np.random.default_rng(2)
    for _ in range(2000):
        a = np.float32(rng.uniform(0.5, 2.0))
        b = np.float32(rng.uniform(0.5, 2.0))
        # c close to -a*b: massive cancellation; the exact product bits decide.
        c = -np.float32(np.float64(a) * np.float64(b))
        _check(a, b, c)
        # c tiny relative to a*b: the exact sum sits near a rounding midpoint.
        c2 = np.float32(np.ldexp(rng.choice([-1.0, 1.0]), -30 + int(rng.integers(-4, 4))))
        _check(a, b, c2)


def test_fma32_differs_from_two_roundings_somewhere():
    # Sanity: the emulation is a real single-rounding fma, not mul-then-add.
    rng = np.random.default_rng(3)
    a = rng.uniform(0.5, 2, 20000).astype(np.float32)
    b = rng.uniform(0.5, 2, 20000).astype(np.float32)
    c = (-(a.astype(np.float64) * b)).astype(np.float32)
    two = (a * b) + c
    one = fma32(a, b, c)
    assert np.any(one != two)


def test_numpy_float32_ops_are_single_rounding():
    rng = np.random.default_rng(4)
    for _ in range(500):
        a, b = (rng.standard_normal(2) * 100).astype(np.float32)
        fa, fb = Fraction(float(a)), Fraction(float(b))
        assert a * b == np.float32(round_to_f32(fa * fb))
        assert a + b == np.float32(round_to_f32(fa + fb)) or (fa + fb) == 0
        assert a / b == np.float32(round_to_f32(fa / fb))
