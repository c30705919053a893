"""Pins for the oracle's error-free transformations, multiword arithmetic and
exact accumulation, checked against exact rationals (``fractions``).

The paper (Section 1) builds DD/TD/QD numbers from 2/3/4 binary64 words; the
algorithms are the published ones named in ``oracle/mwo.c``.  Nothing here
re-types the oracle's formulas: each check is a mathematical property
(exactness of an EFT, an error bound, canonicity, greedy rounding) evaluated
in exact arithmetic.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import exact as X

U = Fraction(1, 2 ** 53)


def _edge_doubles():
    v = [0.0, -0.0, 1.0, -1.0, 0.5, 3.0, 2.0 ** -1074, -(2.0 ** -1074), 2.0 ** -1022,
         2.0 ** -1022 * (1 - 2.0 ** -52), 1.0 + 2.0 ** -52, 1.0 - 2.0 ** -53,
         2.0 ** 52, 2.0 ** 53, 2.0 ** 53 + 2, 2.0 ** 1000, -(2.0 ** 1000), 0.1, 1e300, 1e-300,
         math.pi, -math.e, 2.0 ** -60, 3 * 2.0 ** -54, 2.0 ** -53]
    return v


def _random_doubles(rng, cnt, lo=-60, hi=60):
    m = rng.uniform(-1, 1, cnt)
    e = rng.integers(lo, hi, cnt)
    return np.ldexp(m, e)


def test_twosum_exact_and_rounded():
    rng = np.random.default_rng(1)
    edge = _edge_doubles()
    a = np.array([x for x in edge for _ in edge] + list(_random_doubles(rng, 20000, -300, 300)))
    b = np.array([y for _ in edge for y in edge] + list(_random_doubles(rng, 20000, -300, 300)))
    # exponent gaps from 0 to 1100
    gaps = rng.integers(0, 1100, 5000)
    a2 = rng.uniform(1, 2, 5000) * 2.0 ** 500
    b2 = np.ldexp(rng.uniform(-1, 1, 5000), 500 - gaps)
    a = np.concatenate([a, a2])
    b = np.concatenate([b, b2])
    s, e = oracle.eft(oracle.EFT_TWOSUM, a, b)
    for x, y, ss, ee in zip(a, b, s, e):
        if not (math.isfinite(x + y)):
            continue
        assert ss == x + y
        assert Fraction(x) + Fraction(y) == Fraction(ss) + Fraction(ee)


def test_fasttwosum_exact_under_precondition():
    rng = np.random.default_rng(2)
    a = _random_doubles(rng, 20000, -200, 200)
    b = _random_doubles(rng, 20000, -200, 200)
    big = np.where(np.abs(a) >= np.abs(b), a, b)
    small = np.where(np.abs(a) >= np.abs(b), b, a)
    s, e = oracle.eft(oracle.EFT_FASTTWOSUM, big, small)
    for x, y, ss, ee in zip(big, small, s, e):
        assert ss == x + y
        assert Fraction(x) + Fraction(y) == Fraction(ss) + Fraction(ee)


def test_twoprod_exact_without_underflow():
    rng = np.random.default_rng(3)
    a = _random_doubles(rng, 20000, -400, 400)
    b = _random_doubles(rng, 20000, -400, 400)
    edge = [x for x in _edge_doubles() if x == 0 or 1e-200 < abs(x) < 1e200]
    a = np.concatenate([a, [x for x in edge for _ in edge]])
    b = np.concatenate([b, [y for _ in edge for y in edge]])
    p, e = oracle.eft(oracle.EFT_TWOPROD, a, b)
    for x, y, pp, ee in zip(a, b, p, e):
        if x != 0 and y != 0 and math.frexp(x)[1] + math.frexp(y)[1] < -969:
            continue  # the error term would underflow: excluded by definition
        assert pp == x * y
        assert Fraction(x) * Fraction(y) == Fraction(pp) + Fraction(ee)


def _rand_mw(rng, w, cnt, spread=6, cancel_with=None):
    out = np.zeros((w, cnt))
    for i in range(cnt):
        e = int(rng.integers(-spread, spread + 1))
        v = Fraction(0)
        for k in range(5):
            v += Fraction(int(rng.integers(-2 ** 62, 2 ** 62))) * Fraction(2) ** (e - 62 - 55 * k)
        if cancel_with is not None and i % 2 == 0:
            # y close to -x: heavy cancellation in x + y
            d = Fraction(int(rng.integers(1, 2 ** 20)), 2 ** (20 + int(rng.integers(1, 53 * w + 20))))
            v = -X.words_to_frac(cancel_with[:, i]) * (1 + d)
        out[:, i] = X.greedy_words(v, w)
    return out


# Relative error bounds: DD from Joldes, Muller, Popescu (2017):
# AccurateDWPlusDW 3u^2, DWTimesDW3 <= 5u^2 (proved 4u^2 for the FMA form),
# DWDivDW2 15u^2.  TD/QD (our renormalised forms): addition satisfies the
# weak model |err| <= 2 u^w (|x| + |y|); multiplication and division have
# relative error <= 4 u^w.
@pytest.mark.parametrize("w", [2, 3, 4])
def test_multiword_error_bounds(w):
    rng = np.random.default_rng(10 + w)
    cnt = 1500
    x = _rand_mw(rng, w, cnt)
    y = _rand_mw(rng, w, cnt)
    yc = _rand_mw(rng, w, cnt, cancel_with=x)
    uw = U ** w
    for name, op, yy in (("add", oracle.OP_ADD, y), ("add", oracle.OP_ADD, yc),
                         ("sub", oracle.OP_SUB, y), ("mul", oracle.OP_MUL, y),
                         ("div", oracle.OP_DIV, y)):
        z = oracle.arith(op, w, x, yy)
        for i in range(cnt):
            a = X.words_to_frac(x[:, i])
            b = X.words_to_frac(yy[:, i])
            zz = X.words_to_frac(z[:, i])
            ex = {"add": a + b, "sub": a - b, "mul": a * b, "div": a / b}[name]
            err = abs(zz - ex)
            if w == 2:
                bound = {"add": 3, "sub": 3, "mul": 5, "div": 15}[name] * uw * abs(ex)
            elif name in ("add", "sub"):
                bound = 2 * uw * (abs(a) + abs(b))
            else:
                bound = 4 * uw * abs(ex)
            assert err <= bound, (name, w, i, float(err / abs(ex)) if ex else float(err))


@pytest.mark.parametrize("w", [2, 3, 4])
def test_results_nonoverlapping(w):
    """Result words do not overlap: DD results are canonical (z0 = RN(z0 +
    z1)); TD/QD words stay within one ulp of the word above."""
    rng = np.random.default_rng(20 + w)
    x = _rand_mw(rng, w, 800)
    y = _rand_mw(rng, w, 800)
    for op in (oracle.OP_ADD, oracle.OP_MUL, oracle.OP_DIV):
        z = oracle.arith(op, w, x, y)
        for i in range(z.shape[1]):
            for c in range(w - 1):
                hi, lo = z[c, i], z[c + 1, i]
                if hi == 0:
                    assert lo == 0
                    continue
                assert abs(lo) <= math.ulp(hi), (op, i, c)
            if w == 2:
                assert z[0, i] + z[1, i] == z[0, i]


@pytest.mark.parametrize("w", [2, 3, 4])
def test_exact_cases(w):
    """Operations whose exact result is representable in w words return it
    exactly: small integers, powers of two, x - x = 0, x * 1 = x, x / 1 = x."""
    rng = np.random.default_rng(30 + w)
    cnt = 400
    a = rng.integers(-2 ** 20, 2 ** 20, cnt).astype(float)
    b = rng.integers(1, 2 ** 20, cnt).astype(float)
    x = np.zeros((w, cnt)); x[0] = a
    y = np.zeros((w, cnt)); y[0] = b
    s = oracle.arith(oracle.OP_ADD, w, x, y)
    p = oracle.arith(oracle.OP_MUL, w, x, y)
    for i in range(cnt):
        assert X.words_to_frac(s[:, i]) == Fraction(a[i]) + Fraction(b[i])
        assert X.words_to_frac(p[:, i]) == Fraction(a[i]) * Fraction(b[i])
    xr = _rand_mw(rng, w, cnt)
    one = np.zeros((w, cnt)); one[0] = 1.0
    assert np.array_equal(oracle.arith(oracle.OP_MUL, w, xr, one), xr)
    assert np.array_equal(oracle.arith(oracle.OP_DIV, w, xr, one), xr)
    d = oracle.arith(oracle.OP_SUB, w, xr, xr)
    assert np.all(d == 0)
    # quotient of exactly divisible numbers
    q = oracle.arith(oracle.OP_DIV, w, p, y)
    for i in range(cnt):
        assert X.words_to_frac(q[:, i]) == Fraction(a[i])


@pytest.mark.parametrize("w", [2, 3, 4])
def test_cmpabs_matches_exact_order(w):
    rng = np.random.default_rng(40 + w)
    x = _rand_mw(rng, w, 1000, spread=1)
    # near ties: y = x with a perturbed last word, random sign flips
    y = x.copy()
    y[w - 1] += np.where(rng.random(1000) < 0.5, 1, -1) * np.abs(x[w - 1]) * 2.0 ** -10
    flip = rng.random(1000) < 0.5
    y[:, flip] = -y[:, flip]
    y[:, ::7] = x[:, ::7]          # exact ties
    r = oracle.arith(oracle.OP_CMPABS, w, x, y)
    for i in range(1000):
        a = abs(X.words_to_frac(x[:, i]))
        b = abs(X.words_to_frac(y[:, i]))
        assert r[i] == (a > b) - (a < b), i


def test_exact_sum_greedy_rounding():
    rng = np.random.default_rng(50)
    for trial in range(300):
        cnt = int(rng.integers(1, 60))
        e = rng.integers(-1074, 970, cnt) if trial % 3 == 0 else rng.integers(-200, 200, cnt)
        t = np.ldexp(rng.uniform(-1, 1, cnt), e)
        if trial % 5 == 0:               # exact cancellation pairs
            t = np.concatenate([t, -t[: cnt // 2]])
        if trial % 7 == 0:               # subnormal results
            t = np.array([2.0 ** -1074, 3 * 2.0 ** -1074, -(2.0 ** -1073)] * 3)
        nw = int(rng.integers(1, 9))
        got = oracle.exact_sum(t, nw)
        ref = X.greedy_words(sum((Fraction(v) for v in t), Fraction(0)), nw)
        assert list(got) == ref, (trial, got, ref)


def test_exact_sum_ties_to_even():
    one = 1.0
    ulp_half = 2.0 ** -53
    # 1 + 2^-53 is a tie: rounds to even (1.0); 1 + 3*2^-53 rounds up
    assert oracle.exact_sum([one, ulp_half], 1)[0] == 1.0
    assert oracle.exact_sum([one, 3 * ulp_half], 1)[0] == 1.0 + 2.0 ** -51
    assert oracle.exact_sum([one, ulp_half, 2.0 ** -200], 1)[0] == 1.0 + 2.0 ** -52


def test_exact_dot_products():
    rng = np.random.default_rng(51)
    for trial in range(100):
        cnt = int(rng.integers(1, 80))
        lo, hi = (-500, 500) if trial % 2 else (-40, 40)
        x = np.ldexp(rng.uniform(-1, 1, cnt), rng.integers(lo, hi, cnt))
        y = np.ldexp(rng.uniform(-1, 1, cnt), rng.integers(lo, hi, cnt))
        got = oracle.exact_dot(x, y, 8)
        ref = X.greedy_words(sum((Fraction(a) * Fraction(b) for a, b in zip(x, y)), Fraction(0)), 8)
        assert list(got) == ref
    # products below the TwoProd underflow threshold are still exact
    x = np.array([2.0 ** -1074, 2.0 ** -600, 3.0])
    y = np.array([2.0 ** -1074, 2.0 ** -600, 2.0 ** -1074])
    got = oracle.exact_dot(x, y, 3)
    ref = X.greedy_words(sum((Fraction(a) * Fraction(b) for a, b in zip(x, y)), Fraction(0)), 3)
    assert list(got) == ref


def test_residual_exact_small():
    rng = np.random.default_rng(52)
    for n, wa, wx, wb in ((1, 1, 1, 1), (5, 2, 8, 8), (9, 4, 8, 2), (13, 3, 5, 8)):
        lda = n + 3
        A = np.zeros((wa, n, lda))
        for c in range(wa):
            A[c, :, :n] = np.ldexp(rng.uniform(-1, 1, (n, n)), -55 * c)
        x = np.stack([np.ldexp(rng.uniform(-1, 1, n), -50 * d) for d in range(wx)])
        b = np.stack([np.ldexp(rng.uniform(-1, 1, n), -53 * d) for d in range(wb)])
        r = oracle.residual(A, b, x, 8)
        Af = X.mat_to_frac(A, n)
        xf = X.vec_to_frac(x)
        bf = X.vec_to_frac(b)
        rf = X.residual(Af, bf, xf)
        for i in range(n):
            assert list(r[:, i]) == X.greedy_words(rf[i], 8)
