"""CPU model of the arithmetic behind the FP64-accurate tensor-core products
(exact BF16 slicing, Ozaki scheme): checks, with exact integer arithmetic,
the facts the CUDA kernel relies on.

  * a double scaled by 2^(56 - e) (e = exponent of its row maximum) is an
    integer of at most 57 bits; its balanced base-256 digits
    (q_1 in [-256, 256], q_2..q_7 in [-128, 128]) rebuild it exactly and
    every digit is exact in BF16;
  * the slice products of group g = s + t (g = 2..6) summed over 128 k stay
    below 2^24, so FP32 accumulation of each group is exact;
  * the fixed-point sum I = 2^32 sum_g (group g) grows by less than 2^55.1 per
    128-k drain, so 120 drains stay inside int64;
  * the whole product, with groups g >= 7 accumulated in FP32, is within a
    small multiple of 2^-56 x row max x column max x K of the exact product;
  * the int64 -> double construction (normalise, round to nearest even)
    equals ldexp(float(J), e).
"""
import math
import random

import numpy as np
import pytest

S = 7  # slices per operand


def row_exponent(row):
    """e with max |x| < 2^e (frexp's exponent of the largest entry)."""
    m = max(abs(float(v)) for v in row)
    return math.frexp(m)[1] if m > 0 else None


def digits(x, e):
    """Balanced base-256 digits of round(x 2^(56 - e)), most significant first."""
    X = int(round(math.ldexp(x, 56 - e)))
    q = [0] * S
    for s in range(S - 1, 0, -1):
        d = ((X + 128) & 255) - 128
        q[s] = d
        X = (X - d) >> 8
    q[0] = X
    return q


def test_digits_rebuild_and_bounds():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        row = rng.standard_normal(8) * 10.0 ** rng.uniform(-30, 30, 8)
        e = row_exponent(row)
        for x in row:
            q = digits(float(x), e)
            assert abs(q[0]) <= 256 and all(abs(d) <= 128 for d in q[1:])
            X = sum(d * 256 ** (S - 1 - s) for s, d in enumerate(q))
            assert X == int(round(math.ldexp(float(x), 56 - e)))
            # the row maximum's own bits are kept exactly (2^-56 of the row max below)
            err = abs(math.ldexp(X, e - 56) - float(x))
            assert err <= math.ldexp(1.0, e - 57)
            # every digit scaled by 2^-8(s-1) is exact in BF16 (<= 8 significant bits)
            for d in q:
                assert d == 0 or abs(d) < 2 ** 8 or abs(d) == 256


def test_group_sums_below_2_24():
    """Worst case: every digit at its bound, 128 consecutive k."""
    qmax = [256] + [128] * (S - 1)
    for g in range(2, 7):
        per_k = sum(qmax[s - 1] * qmax[g - s - 1] for s in range(1, g) if 1 <= g - s <= S)
        assert per_k * 128 < 2 ** 24, (g, per_k * 128)


def test_fixed_point_growth_per_drain():
    qmax = [256] + [128] * (S - 1)
    growth = 0
    for g in range(2, 7):
        per_k = sum(qmax[s - 1] * qmax[g - s - 1] for s in range(1, g) if 1 <= g - s <= S)
        growth += per_k * 128 * 2 ** (8 * (6 - g))  # integer of group g shifted by 8 (6 - g)
    assert growth < 2 ** 55.1
    assert 120 * growth < 2 ** 63


def sliced_dot(a, b):
    """The kernel's arithmetic for one output: a (row of op(A)), b (column of
    op(B)); groups 2..6 exact (integers), g >= 7 in FP32; returns
    (value, row max exponent, column max exponent)."""
    ea, eb = row_exponent(a), row_exponent(b)
    qa = [digits(float(x), ea) for x in a]
    qb = [digits(float(x), eb) for x in b]
    K = len(a)
    I = 0
    acc7 = np.float32(0.0)
    for k0 in range(0, K, 128):
        groups = [0] * 7
        for k in range(k0, min(K, k0 + 128)):
            for s in range(1, S + 1):
                for t in range(1, S + 2 - s):
                    g = s + t
                    p = qa[k][s - 1] * qb[k][t - 1]
                    if g <= 6:
                        groups[g - 2] += p
                    else:  # pre-scaled slices: 2^-8(g-2) units, FP32
                        acc7 = np.float32(acc7 + np.float32(p * 2.0 ** (-8 * (g - 2))))
        for g in range(2, 7):
            assert abs(groups[g - 2]) < 2 ** 24
            I += groups[g - 2] << (8 * (6 - g))
    # epilogue: (I + 2^32 acc7) 2^(ea + eb - 48), with acc7 folded into the
    # integer (at 2^-40 while |I| < 2^55, else at 2^-32) and the double built
    # from the integer
    e = ea + eb - 48
    fine = -(1 << 55) < I < (1 << 55)
    t = np.float32(acc7 * np.float32(2.0 ** (40 if fine else 32)))
    add = int(round(float(t)))  # round half to even, as the float -> int conversion
    if fine:
        J, e = I * 256 + add, e - 8
    else:
        J = I + add
    return fix_to_double(J, e), ea, eb


@pytest.mark.parametrize("K", [64, 200])
def test_sliced_product_error_bound(K):
    from fractions import Fraction
    rng = np.random.default_rng(K)
    for _ in range(6):
        a = rng.standard_normal(K) * 10.0 ** rng.uniform(-8, 8, K)
        b = rng.standard_normal(K) * 10.0 ** rng.uniform(-8, 8, K)
        val, ea, eb = sliced_dot(a, b)
        exact = sum(Fraction(float(x)) * Fraction(float(y)) for x, y in zip(a, b))
        err = abs(Fraction(val) - exact)
        bound = Fraction(4 * K) * Fraction(2) ** (ea + eb - 56)
        assert err <= bound, (float(err), float(bound))


def fix_to_double(J, e):
    """Integer construction of J 2^e as a double (round to nearest even)."""
    if J == 0:
        return 0.0
    sgn = J < 0
    mag = -J if sgn else J
    lz = 64 - mag.bit_length()
    m = mag << lz
    mant, rem = m >> 11, m & 0x7FF
    E = 63 - lz + e
    if rem > 0x400 or (rem == 0x400 and (mant & 1)):
        mant += 1
        if mant >> 53:
            mant >>= 1
            E += 1
    if E < -1022 or E > 1023:
        return math.ldexp(float(J), e)
    v = math.ldexp(mant, E - 52)
    return -v if sgn else v


def test_fix_to_double_matches_ldexp():
    rnd = random.Random(7)
    for _ in range(200000):
        bits = rnd.randint(1, 63)
        J = rnd.getrandbits(bits)
        if rnd.random() < 0.3:  # exact ties and near ties of the 11 dropped bits
            J = ((J >> 11) << 11) | rnd.choice([0x3FF, 0x400, 0x401])
        if rnd.random() < 0.5:
            J = -J
        e = rnd.randint(-1100, 960)  # results up to the largest finite doubles
        assert fix_to_double(J, e) == math.ldexp(float(J), e)
