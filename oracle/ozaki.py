"""Oracle for the split-precision slab product of the DD trailing update
and the standalone DD block product: C -= L U (or C += L U) for one slab of
K <= 64 inner terms, computed by Ozaki's scheme I (error-free splitting of
the operands into short integer digits whose pairwise products are exact;
Ozaki, Ogita, Oishi and Rump, Numer. Algorithms 59 (2012)), in the form the
GPU path implements.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Python integers and
fractions throughout; numpy only for the exact integer digit products.

The method, for an m x K row operand L, a K x N column operand U and the
m x N DD matrix C (all DD: word 0 hi, word 1 lo):

1. Scales.  e_i = ilogb(max_t |hi(l_it)|) + 2 for row i of L, f_j likewise
   over column j of U (0 for an all-zero row or column), so every scaled
   entry lies in (-1/2, 1/2).
2. Integers.  An entry x = hi + lo of row i becomes
   X = floor(hi 2^(120 - e_i)) + floor(lo 2^(120 - e_i))
   (the two words floored separately); columns of U likewise with f_j.
3. Digits.  X = sum_{p=1..15} a_p 256^(15 - p): the 14 low digits balanced
   in [-128, 127] (taken from the least significant end), a_1 the rest.
4. Diagonals.  D_d = sum_{p + q = d} sum_t a_p(i, t) b_q(t, j) for
   d = 2..16 (pairs with p + q > 16 are dropped); exact integers.
5. Product.  R = sum_d D_d 2^(8 (16 - d)); the slab product is P = R 2^s
   with s = e_i + f_j - 128.
6. Result, exact form: when both words of C are integer multiples of 2^s
   of magnitude below 2^(s + 158), V = C - P (C + P) is formed exactly and
   rounded greedily: hi = RN(V), lo = RN(V - hi); a zero V or remainder
   gives +0.  This form is taken when hi and lo come out normal (or zero).
7. Result, otherwise: P is rounded greedily to a DD pair and subtracted
   from (added to) C with the library's DD arithmetic (the oracle's
   ``OP_SUB`` / ``OP_ADD``).

Products in the subnormal range are outside this model (the GPU rounds them
twice in step 7); the tests use normal-range data.

Arrays follow the package conventions: word c of X(i, j) at X[c, j, i].
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

from . import OP_ADD, OP_SUB, arith

NDIG = 15          # digits per operand
MAXD = 16          # largest digit-order sum kept
GRID = 120         # scaled entries are floored onto 2^-GRID
WIDTH = 158        # C words below 2^(s + WIDTH) take the exact form
TWO = Fraction(2)


def _ilogb(v: float) -> int:
    return math.frexp(v)[1] - 1


def scale_exponent(hi_words) -> int:
    """ilogb(max |hi|) + 2, or 0 when every word is zero (step 1)."""
    mx = max((abs(float(v)) for v in hi_words), default=0.0)
    return _ilogb(mx) + 2 if mx != 0.0 else 0


def floor_scaled(v: float, sh: int) -> int:
    """floor(v 2^sh) for a finite double v (exact)."""
    q = Fraction(v) * TWO ** sh
    return math.floor(q)


def digits(X: int):
    """The 15 base-256 digits of X, most significant first (step 3)."""
    a = [0] * NDIG
    for p in range(NDIG - 1, 0, -1):
        d = X & 0xFF
        if d >= 128:
            d -= 256
        a[p] = d
        X = (X - d) >> 8
    a[0] = X
    return a


def _rn(v: Fraction) -> float:
    return float(v)      # correctly rounded to nearest, ties to even


def _normal_or_zero(x: float) -> bool:
    return x == 0.0 or (math.isfinite(x) and abs(x) >= 2.0 ** -1022)


def slab_product(L: np.ndarray, U: np.ndarray, m: int, N: int, K: int):
    """(R, e, f) for L (2, K, >= m) and U (2, N, >= K): R[i][j] the exact
    integer of step 5, e and f the row and column scales."""
    e = [scale_exponent(L[0, :K, i]) for i in range(m)]
    f = [scale_exponent(U[0, j, :K]) for j in range(N)]
    A = np.zeros((NDIG, m, K), dtype=np.int64)
    B = np.zeros((NDIG, K, N), dtype=np.int64)
    for i in range(m):
        for t in range(K):
            X = floor_scaled(L[0, t, i], GRID - e[i]) + floor_scaled(L[1, t, i], GRID - e[i])
            A[:, i, t] = digits(X)
    for j in range(N):
        for t in range(K):
            X = floor_scaled(U[0, j, t], GRID - f[j]) + floor_scaled(U[1, j, t], GRID - f[j])
            B[:, t, j] = digits(X)
    D = {}
    for p in range(1, NDIG + 1):
        for q in range(1, NDIG + 1):
            if p + q <= MAXD:
                D[p + q] = D.get(p + q, 0) + A[p - 1] @ B[q - 1]
    R = [[sum(int(D[d][i, j]) << (8 * (MAXD - d)) for d in range(2, MAXD + 1)) for j in range(N)]
         for i in range(m)]
    return R, e, f


def update(C: np.ndarray, L: np.ndarray, U: np.ndarray, m: int, N: int, K: int, plus: bool = False):
    """C -= L U (plus: C += L U) for one slab by steps 1-7; returns the new
    (2, N, m) array and the count of entries that took the exact form."""
    R, e, f = slab_product(L, U, m, N, K)
    out = np.zeros((2, N, m))
    fallback_c, fallback_p = [], []
    where = []
    exact_count = 0
    for i in range(m):
        for j in range(N):
            s = e[i] + f[j] - 128
            c0, c1 = float(C[0, j, i]), float(C[1, j, i])
            P = R[i][j] * TWO ** s
            words_ok = all(w == 0.0 or ((Fraction(w) / TWO ** s).denominator == 1
                                        and abs(Fraction(w)) < TWO ** (s + WIDTH))
                           for w in (c0, c1))
            done = False
            if words_ok:
                V = Fraction(c0) + Fraction(c1) + (P if plus else -P)
                try:
                    hi = _rn(V)
                    lo = _rn(V - Fraction(hi))
                except OverflowError:
                    hi = lo = math.inf
                if _normal_or_zero(hi) and _normal_or_zero(lo):
                    out[0, j, i] = hi + 0.0       # +0 for a zero result
                    out[1, j, i] = lo + 0.0
                    exact_count += 1
                    done = True
            if not done:
                ph = _rn(P)
                pl = _rn(P - Fraction(ph))
                fallback_c.append((c0, c1))
                fallback_p.append((ph, pl))
                where.append((i, j))
    if where:
        cc = np.array(fallback_c).T.copy()
        pp = np.array(fallback_p).T.copy()
        res = arith(OP_ADD if plus else OP_SUB, 2, cc, pp)
        for k, (i, j) in enumerate(where):
            out[:, j, i] = res[:, k]
    return out, exact_count
