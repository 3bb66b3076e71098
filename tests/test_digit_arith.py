"""The float32 arithmetic of the digit split and of the group combination that
the tensor-core kernels use (Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59,
2012), emulated in numpy with every operation rounded to float32, and checked
against facts that do not depend on it: the digits rebuild the value to
within 2^(E-45), they are small integers times their weights (exact in bf16),
the weighted split gives the same digits as the split that rescales the
remainder at every step, and the TwoSum combination of integer group sums is
accurate to df64 against an exact rational sum. No GPU is used."""
from fractions import Fraction

import numpy as np

f32 = np.float32


def _split_weighted(h, l, E, N=7):
    """d[i] = d_i 2^(-7 i): magic constant 1.5 * 2^(23 - 7i) rounds the
    remainder to the digit's grid; the remainder is never rescaled."""
    s = f32(2.0 ** (7 - E))
    a, b = f32(h * s), f32(l * s)
    d = []
    for i in range(N):
        if i == 3:
            a = f32(a + b)
        m = f32(12582912.0 * 2.0 ** (-7 * i))
        di = f32(f32(a + m) - m)
        d.append(di)
        a = f32(a - di)
    return d


def _split_rescaled(h, l, E, N=7):
    """Integer digits d_i: rint by the magic constant 1.5 * 2^23, then the
    remainder is scaled up by 128 (l folded in at digit 3, pre-scaled by 2^21)."""
    s = f32(2.0 ** (7 - E))
    a, b = f32(h * s), f32(f32(l * s) * f32(2.0 ** 21))
    d = []
    for i in range(N):
        if i == 3:
            a = f32(a + b)
        di = f32(f32(a + f32(12582912.0)) - f32(12582912.0))
        d.append(di)
        a = f32(f32(a - di) * f32(128.0))
    return d


def _two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def _combine_weighted(S):
    """sum of weighted group sums S[g] (= integer * 2^(-7 g)) as hi + lo"""
    h, l = S[-1], f32(0.0)
    for g in range(len(S) - 2, -1, -1):
        h, e = _two_sum(S[g], h)
        l = f32(l + e)
    s = f32(h + l)
    return s, f32(l - f32(s - h))


def _samples(rng, count):
    for _ in range(count):
        x = rng.standard_normal() * 10.0 ** rng.uniform(-25, 25)
        h = f32(x)
        l = f32(x - float(h))
        # column exponent: at or above the value's own (the column maximum may be larger)
        E = int(np.floor(np.log2(abs(float(h))))) + 1 + int(rng.integers(0, 4))
        yield h, l, E


def test_digits_rebuild_the_value_on_the_grid():
    """x - sum_i d_i 2^(E-7) is the remainder below the last digit's grid
    (at most half of 2^(E-49)) plus the one float32 rounding where l joins
    the remainder after digit 2 (at most half an ulp of a number below
    2^(E-22): 2^(E-46)); together under 2^(E-45)."""
    rng = np.random.default_rng(11)
    for h, l, E in _samples(rng, 4000):
        d = _split_weighted(h, l, E)
        x = Fraction(float(h)) + Fraction(float(l))
        rebuilt = sum(Fraction(float(di)) for di in d) * Fraction(2) ** (E - 7)
        assert abs(x - rebuilt) <= Fraction(2) ** (E - 46) + Fraction(2) ** (E - 50), (h, l, E)


def test_digits_are_small_integers_exact_in_bf16():
    rng = np.random.default_rng(12)
    for h, l, E in _samples(rng, 4000):
        for i, di in enumerate(_split_weighted(h, l, E)):
            k = float(di) * 2.0 ** (7 * i)
            assert k == int(k) and abs(k) <= (128 if i == 0 else 72), (i, k)
            # bf16 keeps the upper 16 bits of a float32
            assert np.frombuffer(np.float32(di).tobytes(), np.uint32)[0] & 0xFFFF == 0


def test_weighted_split_equals_rescaled_split():
    rng = np.random.default_rng(13)
    for h, l, E in _samples(rng, 4000):
        w = _split_weighted(h, l, E)
        r = _split_rescaled(h, l, E)
        for i in range(7):
            assert w[i] == f32(r[i] * f32(2.0 ** (-7 * i))), (h, l, E, i)


def test_combination_is_df64_accurate():
    """Integer group sums below 2^24, carried with their weights 2^(-7 g):
    hi + lo is within 2^-46 of the exact sum (relative), 7 and 6 groups."""
    rng = np.random.default_rng(14)
    for trial in range(3000):
        N = 7 if trial % 2 else 6
        lim = 2 ** 23 if trial % 3 else 300
        ints = [int(v) for v in rng.integers(-lim, lim, N)]
        S = [f32(k * 2.0 ** (-7 * g)) for g, k in enumerate(ints)]
        assert all(Fraction(float(S[g])) == Fraction(ints[g]) * Fraction(2) ** (-7 * g) for g in range(N))
        hi, lo = _combine_weighted(S)
        exact = sum(Fraction(k) * Fraction(2) ** (-7 * g) for g, k in enumerate(ints))
        got = Fraction(float(hi)) + Fraction(float(lo))
        assert abs(got - exact) <= Fraction(2) ** -46 * abs(exact) + Fraction(2) ** -60, (ints, got, exact)
