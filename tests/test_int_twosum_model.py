"""The integer TwoSum of the device arithmetic (mw_arith.cuh: the two
significands aligned into a 128-bit integer, added exactly, rounded to
nearest-even, the remainder as the error word), restated here in Python
integers and checked against Knuth's six-operation TwoSum in binary64
(Python floats round to nearest-even) on random and edge-case pairs.

This pins the algorithm's steps on the CPU; the GPU tests then check the
device code itself bitwise against the oracle's arithmetic."""
import math
import random
import struct

MAN = (1 << 52) - 1
HID = 1 << 52
SIGN = 1 << 63


def bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def dbl(b):
    return struct.unpack("<d", struct.pack("<Q", b & ((1 << 64) - 1)))[0]


def knuth(a, b):
    s = a + b
    av = s - b
    bv = s - av
    return s, (a - av) + (b - bv)


def pack(r, E, sg):
    L = r.bit_length()
    Ee = E + (L - 53)
    if Ee < 1 or Ee > 2046:
        return None
    m = (r >> (L - 53)) if L >= 53 else (r << (53 - L))
    return dbl(sg | (Ee << 52) | (m & MAN))


def sum_ordered(A, B):
    """(s, e) for bit patterns with |a| >= |b|, or None (fall back)."""
    ua, ub = A & ~SIGN, B & ~SIGN
    ea, eb = ua >> 52, ub >> 52
    if ea == 2047:
        return None
    if ub == 0:
        return dbl(A if ua else (A & B & SIGN)), 0.0
    if eb == 0:
        return None
    d = ea - eb
    if d > 54:
        return dbl(A), dbl(B)
    sa = A & SIGN
    ma, mb = (ua & MAN) | HID, (ub & MAN) | HID
    M = (ma << d) - mb if (A ^ B) & SIGN else (ma << d) + mb
    if M == 0:
        return 0.0, 0.0
    L = M.bit_length()
    if L <= 53:
        s = pack(M, eb, sa)
        return None if s is None else (s, 0.0)
    sh = L - 53
    q, r = M >> sh, M & ((1 << sh) - 1)
    half = 1 << (sh - 1)
    up = r > half or (r == half and q & 1)
    Es = eb + sh
    rem = r - ((1 << sh) if up else 0)
    if up:
        q += 1
        if q == 1 << 53:
            q >>= 1
            Es += 1
    if Es > 2046:
        return None
    s = dbl(sa | (Es << 52) | (q & MAN))
    if rem == 0:
        return s, 0.0
    e = pack(abs(rem), eb, (sa ^ SIGN) if rem < 0 else sa)
    return None if e is None else (s, e)


def int_two_sum(a, b):
    A, B = bits(a), bits(b)
    if (A << 1) & ((1 << 64) - 1) < (B << 1) & ((1 << 64) - 1):
        A, B = B, A
    r = sum_ordered(A, B)
    return knuth(a, b) if r is None else r


def _same(x, y):
    return bits(x) == bits(y) or (math.isnan(x) and math.isnan(y))


def _cases(rng, cnt):
    for _ in range(cnt):
        k = rng.randrange(8)
        a = rng.uniform(-1, 1) * 2.0 ** rng.randrange(-40, 40)
        if k == 0:
            b = rng.uniform(-1, 1) * 2.0 ** rng.randrange(-40, 40)
        elif k == 1:                                    # exponent gaps around the cut at 55
            b = math.copysign(rng.uniform(0.5, 1.0), rng.choice([-1, 1])) * 2.0 ** (math.frexp(a)[1] - rng.randrange(50, 60))
        elif k == 2:                                    # near cancellation
            b = -math.nextafter(a, rng.choice([math.inf, -math.inf]))
        elif k == 3:                                    # halfway cases, also below a power of two
            a = math.copysign(2.0 ** rng.randrange(-20, 20), rng.choice([-1, 1])) if rng.random() < 0.5 else a
            b = rng.choice([-1, 1]) * math.ulp(a) * rng.choice([0.25, 0.5, 0.75, 1.0, 1.5])
        elif k == 4:                                    # zeros (either side, both signs) and exact cancellation
            b = rng.choice([0.0, -0.0, -a])
            if rng.random() < 0.3:
                a = rng.choice([0.0, -0.0])
        elif k == 5:                                    # subnormal words
            a = rng.choice([5e-324, -5e-324, 2.2250738585072014e-308, 1e-310])
            b = rng.choice([-5e-324, 3e-310, -2.2250738585072014e-308])
        elif k == 6:                                    # near overflow
            a = rng.choice([1.7e308, -1.7e308, 8.98846567431158e307])
            b = rng.choice([1.7e308, 8.98846567431158e307, -1.0])
        else:                                           # DD-shaped pairs
            b = a * 2.0 ** -53 * rng.uniform(-1, 1)
        yield a, b


def test_int_two_sum_model_matches_knuth():
    rng = random.Random(2107)
    n = 0
    for a, b in _cases(rng, 60000):
        s1, e1 = int_two_sum(a, b)
        s2, e2 = knuth(a, b)
        assert _same(s1, s2) and _same(e1, e2), (a, b, (s1, e1), (s2, e2))
        n += 1
    assert n == 60000


def test_int_two_sum_model_fast_path_is_exact():
    """On the integer path s + e equals a + b exactly and s = RN(a + b)."""
    from fractions import Fraction
    rng = random.Random(12550)
    hits = 0
    for a, b in _cases(rng, 5000):
        A, B = bits(a), bits(b)
        if (A << 1) & ((1 << 64) - 1) < (B << 1) & ((1 << 64) - 1):
            A, B = B, A
        r = sum_ordered(A, B)
        if r is None:
            continue
        hits += 1
        s, e = r
        assert Fraction(s) + Fraction(e) == Fraction(a) + Fraction(b)
        assert s == a + b
    assert hits > 3000
