"""The 61-bit fixed-point arithmetic of the mixed handover transform (k_transform_from_q), emulated with
Python integers operation by operation (64-bit two's complement, arithmetic shifts, 32-bit limbs) and
checked against exact rational arithmetic: the conversion from double truncates by less than 2^-61,
a product errs by less than 3 * 2^-61 and never leaves the 64-bit range for factors of magnitude <= 1,
and the conversion back to double is correctly rounded to nearest. CPU only."""
import random
import struct
from fractions import Fraction

MASK64 = (1 << 64) - 1


def dbits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def bdouble(b):
    return struct.unpack("<d", struct.pack("<Q", b & MASK64))[0]


def to_q61(x):
    b = dbits(x)
    ed = (b >> 52) & 0x7FF
    m = (b & ((1 << 52) - 1)) | (1 << 52)
    sh = ed - 1014
    q = (m << (sh & 15)) if sh >= 0 else ((m >> (-sh)) if sh > -64 else 0)
    if ed == 0:
        q = 0
    return -q if (b >> 63) else q


def from_q61(q):
    if q == 0:
        return 0.0
    sign = 1 << 63 if q < 0 else 0
    m = -q if q < 0 else q
    lz = 64 - m.bit_length()
    m = (m << lz) & MASK64
    mant, rest = m >> 11, m & 0x7FF
    if rest > 0x400 or (rest == 0x400 and (mant & 1)):
        mant += 1
    e = 2 - lz
    if mant >> 53:
        mant >>= 1
        e += 1
    return bdouble(sign | ((e + 1023) << 52) | (mant & ((1 << 52) - 1)))


def mul_q61(a, b):
    ah, bh = a >> 31, b >> 31  # signed high limbs
    al, bl = a & 0x7FFFFFFF, b & 0x7FFFFFFF  # 31-bit low limbs
    for limb in (ah, bh, al, bl):
        assert -(1 << 31) <= limb < (1 << 31)  # each a 32-bit signed operand
    cross = ah * bl + al * bh
    assert -(1 << 63) <= cross < (1 << 63)
    r = ((ah * bh) << 1) + (cross >> 30)
    assert -(1 << 63) <= r < (1 << 63)
    return r


def test_to_q61_truncates_below_one_unit():
    rng = random.Random(1)
    for _ in range(20000):
        x = rng.uniform(-1.0, 1.0) * 2.0 ** -rng.randint(0, 40)
        assert abs(Fraction(to_q61(x), 2 ** 61) - Fraction(x)) < Fraction(1, 2 ** 61)
    for x in (1.0, -1.0, 0.0, 2.0 ** -70):
        assert abs(Fraction(to_q61(x), 2 ** 61) - Fraction(x)) < Fraction(1, 2 ** 61)


def test_product_error_and_range():
    rng = random.Random(2)
    worst = Fraction(0)
    for _ in range(20000):
        x, y = rng.uniform(-1, 1), rng.uniform(-1, 1)
        if rng.random() < 0.05:
            x = rng.choice([1.0, -1.0, 0.0, 1.0 + 2.0 ** -52])
        qx, qy = to_q61(x), to_q61(y)
        exact = Fraction(qx, 2 ** 61) * Fraction(qy, 2 ** 61)
        worst = max(worst, abs(Fraction(mul_q61(qx, qy), 2 ** 61) - exact) * 2 ** 61)
    assert worst < 3


def test_sum_of_unit_row_products_stays_in_range():
    """An entry of a product of two SU(3)-like matrices: sum_k a_k b_k of unit complex 3-vectors, with every
    partial sum of the real and imaginary parts below 2^62 in Q61."""
    rng = random.Random(3)
    for _ in range(2000):
        v = [complex(rng.gauss(0, 1), rng.gauss(0, 1)) for _ in range(6)]
        na = sum(abs(z) ** 2 for z in v[:3]) ** 0.5
        nb = sum(abs(z) ** 2 for z in v[3:]) ** 0.5
        a, b = [z / na for z in v[:3]], [z / nb for z in v[3:]]
        re = im = 0
        for ak, bk in zip(a, b):
            ar, ai, br, bi = (to_q61(t) for t in (ak.real, ak.imag, bk.real, bk.imag))
            for step in (mul_q61(ar, br), -mul_q61(ai, bi)):
                re += step
                assert abs(re) < 1 << 62
            for step in (mul_q61(ar, bi), mul_q61(ai, br)):
                im += step
                assert abs(im) < 1 << 62


def test_conversion_to_double_is_correctly_rounded():
    rng = random.Random(4)
    for _ in range(50000):
        q = rng.randint(-(1 << 62), 1 << 62) >> rng.randint(0, 60)
        assert from_q61(q) == float(Fraction(q, 2 ** 61))
    for q in (1, -1, 1 << 61, -(1 << 61), (1 << 62) - 1, 0x400 | (1 << 61)):
        assert from_q61(q) == float(Fraction(q, 2 ** 61))
