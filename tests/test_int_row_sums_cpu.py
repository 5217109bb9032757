"""The arithmetic of the integer row sums that GS(1) and GS(2) use on FP64
rows (device_common.cuh: row_int_sum, int_sum_to_double), restated with
Python integers and checked against exact rational sums: every entry's
53-bit significand aligned to the row's largest exponent, |a| with 48
guard bits in a 128-bit accumulator, a^2 as the square of the significand
shifted with 5 guard bits, one rounding to double at the end.  The GPU
parity tests check the CUDA code itself against the oracle; this test pins
the design (alignment units, guard bits, accumulator width, rounding) that
the code implements, so that a wrong unit or a missing guard bit shows up
here as a result off by more than an ulp.  The sum before its rounding is
the exact one to within len 2^-55 (bits shifted out below the unit), so the
double is the correctly rounded sum or its neighbour, and exactly the
correctly rounded one when no bit is shifted out."""
import random
import struct
from fractions import Fraction

MASK128 = (1 << 128) - 1


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def _from_bits(b):
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def _to_double(acc, unit_exp):
    lead = acc.bit_length() - 1
    shift = lead - 52
    if shift <= 0:
        mant = acc << (-shift)
    else:
        mant = acc >> shift
        rem, half = acc & ((1 << shift) - 1), 1 << (shift - 1)
        if rem > half or (rem == half and (mant & 1)):
            mant += 1
            if mant >> 53:
                mant >>= 1
                shift += 1
    return _from_bits(((shift + unit_exp + 52 + 1023) << 52) | (mant & ((1 << 52) - 1)))


def _row_int_sum(v, squares):
    bs = [_bits(x) & 0x7FFFFFFFFFFFFFFF for x in v]
    emax = max(bs) >> 52
    acc = 0
    for b in bs:
        e = b >> 52
        m = (b & ((1 << 52) - 1)) | ((e != 0) << 52)
        d = emax - (e if e else 1)
        if squares:
            if d < 58:
                q = ((m << 5) >> d) & ((1 << 64) - 1)
                acc += q * q
        elif d < 101:
            acc += ((m << 48) >> d) & MASK128
        assert acc <= MASK128  # the accumulator never overflows 128 bits
    return _to_double(acc, 2 * emax - 2160 if squares else emax - 1123)


def test_integer_row_sums_are_correctly_rounded():
    rng = random.Random(20240611)
    for _ in range(4000):
        n = rng.randint(1, 12)
        e0 = rng.randint(-470, 470)
        spread = rng.choice([0, 3, 20, 60, 200])
        v = [rng.choice([-1.0, 1.0]) * rng.uniform(1, 2) * 2.0 ** (e0 + rng.randint(-spread, 0)) for _ in range(n)]
        if n > 1 and rng.random() < 0.1:
            v[0] = 0.0
        emax = max(_bits(abs(x)) >> 52 for x in v) - 1023
        for squares in (False, True):
            if abs(emax) >= (480 if squares else 1000):
                continue  # those rows take the FP64 route on the device
            exact = sum((Fraction(x) ** 2 if squares else abs(Fraction(x))) for x in v)
            got = _row_int_sum(v, squares)
            assert abs(Fraction(got) - exact) < Fraction(1, 2**52) * exact, (v, squares)  # within an ulp
            if len({_bits(abs(x)) >> 52 for x in v if x}) == 1:  # nothing shifted out: exact, one rounding
                assert got == float(exact), (v, squares)  # float(Fraction) rounds to nearest


def test_longest_rows_fit_the_accumulator():
    # 4,095 entries of the largest significand (the a^2 limit) and 2^20 - 1
    # (the |a| limit, summed here in closed form) stay within 128 bits
    top = (1 << 53) - 1
    assert 4095 * ((top << 5) ** 2) <= MASK128
    assert ((1 << 20) - 1) * (top << 48) <= MASK128
    v = [1.9999999999999998] * 4095
    assert _row_int_sum(v, True) == float(4095 * Fraction(1.9999999999999998) ** 2)
