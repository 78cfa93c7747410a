"""Exact-arithmetic check of the two FP32 roundings that the LJ kernel uses to
turn a force component v (in 2^-13 kJ/mol/nm units) into an integer
(reading 18 of the design notes; the kernel itself is checked on the GPU
against the oracle and by the exact zero net force of the pairwise mode).

- one FFMA with the offset M = 1.5 * 2^23: bits(v + M) - bits(M) = rint(v)
  (ties to even) for |v| < 2^22;
- the pairwise-exact form: t = fma(v, 2^-8, M), hi = t - M,
  r = fma(hi, -256, v), l = r + M; (bits(t) << 8) + bits(l) minus the
  constant (bits(M) << 8) + bits(M) is rint(v) for |v| < 2^30.

Every FP32 operation is modelled as the exact rational result rounded once to
the nearest FP32 number, ties to even (IEEE 754 binary32, normal range), with
Python fractions, so no step here depends on the host's floating point.
"""
import random
import struct
from fractions import Fraction

M = Fraction(3 * 2**22)   # 1.5 * 2^23


def rint_even(x: Fraction) -> int:
    f = x.numerator // x.denominator
    d = x - f
    if d > Fraction(1, 2) or (d == Fraction(1, 2) and f % 2 == 1):
        return f + 1
    return f


def round_f32(x: Fraction) -> Fraction:
    """x rounded to the nearest binary32 number (ties to even); normal range."""
    if x == 0:
        return Fraction(0)
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    ulp = Fraction(2) ** (e - 23)
    return rint_even(x / ulp) * ulp


def bits_f32(x: Fraction) -> int:
    return struct.unpack("<I", struct.pack("<f", float(x)))[0]


def one_ffma(v: Fraction) -> int:
    return bits_f32(round_f32(v + M)) - bits_f32(M)


def two_part(v: Fraction) -> int:
    t = round_f32(v * Fraction(1, 256) + M)
    hi = round_f32(t - M)
    r = round_f32(hi * -256 + v)
    lo = round_f32(r + M)
    off = ((bits_f32(M) << 8) + bits_f32(M)) & 0xFFFFFFFF
    q = (((bits_f32(t) << 8) + bits_f32(lo)) - off) & 0xFFFFFFFF
    return q - 2**32 if q >= 2**31 else q


def f32_values(n, lo_exp, hi_exp, seed):
    rng = random.Random(seed)
    out = []
    for _ in range(n):
        e = rng.randint(lo_exp, hi_exp)
        m = rng.randint(2**23, 2**24 - 1)
        v = Fraction(m) * Fraction(2) ** (e - 23)
        out.append(v if rng.random() < 0.5 else -v)
    # ties, neighbours of ties, integers, values next to the range limits
    for k in (0, 1, 2, 3, 1001, 2**20 + 1):
        for s in (1, -1):
            out += [s * (Fraction(k) + Fraction(1, 2)), s * Fraction(k), s * (Fraction(k) + Fraction(1, 4))]
    return out


def test_one_ffma_offset_rounds_to_the_nearest_integer():
    for v in f32_values(3000, -12, 21, seed=1):
        assert round_f32(v) == v
        assert one_ffma(v) == rint_even(v), v
    # just below 2^22 in magnitude
    top = Fraction(2**22) - Fraction(1, 2)
    assert one_ffma(top) == rint_even(top) and one_ffma(-top) == rint_even(-top)


def test_two_part_rounding_is_exact_up_to_2_30():
    for v in f32_values(3000, -12, 29, seed=2):
        assert round_f32(v) == v
        assert two_part(v) == rint_even(v), v
    big = Fraction(2**30) - Fraction(2**6)   # the largest binary32 below 2^30
    assert two_part(big) == rint_even(big) and two_part(-big) == rint_even(-big)


def test_two_part_rounding_gives_opposite_integers_for_opposite_values():
    # the pairwise mode adds +q to i and -q to j: rint is odd, so the two
    # atoms' integers cancel exactly
    for v in f32_values(1000, -4, 29, seed=3):
        assert two_part(-v) == -two_part(v)
