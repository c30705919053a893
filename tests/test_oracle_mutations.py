"""Planted mistakes: each test compiles a copy of the oracle with one
plausible error (a dropped term, a wrong sign, a wrong index or tie rule)
and shows that a pin rejects it, while the unmodified oracle passes the
same pin.  Mistakes are planted in the oracle only, on the CPU."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import exact as X
from paper_2107_12550_gb300 import workloads as W

U = Fraction(1, 2 ** 53)


def _rand_mw(rng, w, cnt):
    out = np.zeros((w, cnt))
    for i in range(cnt):
        v = Fraction(0)
        for k in range(5):
            v += Fraction(int(rng.integers(-2 ** 62, 2 ** 62))) * Fraction(2) ** (-62 - 55 * k)
        out[:, i] = X.greedy_words(v, w)
    return out


def pin_dd_mul():
    rng = np.random.default_rng(1)
    x, y = _rand_mw(rng, 2, 200), _rand_mw(rng, 2, 200)
    z = oracle.arith(oracle.OP_MUL, 2, x, y)
    return all(abs(X.words_to_frac(z[:, i]) - X.words_to_frac(x[:, i]) * X.words_to_frac(y[:, i]))
               <= 5 * U ** 2 * abs(X.words_to_frac(x[:, i]) * X.words_to_frac(y[:, i]))
               for i in range(200))


def pin_add(w):
    def f():
        rng = np.random.default_rng(2)
        x, y = _rand_mw(rng, w, 200), _rand_mw(rng, w, 200)
        z = oracle.arith(oracle.OP_ADD, w, x, y)
        for i in range(200):
            a, b = X.words_to_frac(x[:, i]), X.words_to_frac(y[:, i])
            bound = (3 * U ** 2 * abs(a + b)) if w == 2 else 2 * U ** w * (abs(a) + abs(b))
            if abs(X.words_to_frac(z[:, i]) - (a + b)) > bound:
                return False
        return True
    return f


def pin_twoprod():
    rng = np.random.default_rng(3)
    a, b = rng.uniform(-1, 1, 500), rng.uniform(-1, 1, 500)
    p, e = oracle.eft(oracle.EFT_TWOPROD, a, b)
    return all(Fraction(x) * Fraction(y) == Fraction(pp) + Fraction(ee)
               for x, y, pp, ee in zip(a, b, p, e))


def pin_twosum():
    """TwoSum is exact for any pair: s + e = a + b, with s = RN(a + b); the
    pairs span exponent gaps in both orders."""
    rng = np.random.default_rng(11)
    a = rng.uniform(-1, 1, 500) * 2.0 ** rng.integers(-60, 60, 500)
    b = rng.uniform(-1, 1, 500) * 2.0 ** rng.integers(-60, 60, 500)
    s, e = oracle.eft(oracle.EFT_TWOSUM, a, b)
    return all(Fraction(x) + Fraction(y) == Fraction(ss) + Fraction(ee) and ss == x + y
               for x, y, ss, ee in zip(a, b, s, e))


def pin_fasttwosum():
    """FastTwoSum is exact when the exponent of a is at least that of b."""
    rng = np.random.default_rng(12)
    a = rng.uniform(1, 2, 500) * 2.0 ** rng.integers(0, 40, 500)
    b = rng.uniform(-1, 1, 500)
    s, e = oracle.eft(oracle.EFT_FASTTWOSUM, a, b)
    return all(Fraction(x) + Fraction(y) == Fraction(ss) + Fraction(ee) for x, y, ss, ee in zip(a, b, s, e))


def pin_lu_ties():
    A = np.zeros((2, 3, 3))
    M = [[1.0, 2.0, 3.0], [-1.0, 5.0, 1.0], [1.0, 1.0, 7.0]]
    for i in range(3):
        for j in range(3):
            A[0, j, i] = M[i][j]
    _, piv, _ = oracle.lu(2, A)
    return piv[0] == 0


def pin_lu_factors():
    # P A = L U exactly with dyadic factors; the computed factors must be exact
    n = 6
    rng = np.random.default_rng(4)
    L = np.eye(n) + np.tril(rng.integers(-7, 8, (n, n)) / 8.0, -1)
    Um = np.triu(rng.integers(-9, 10, (n, n)).astype(float)) + 10 * np.eye(n)
    M = L @ Um
    A = np.zeros((2, n, n))
    A[0] = M.T
    LU, piv, info = oracle.lu(2, A)
    got = LU[0].T
    ref = np.tril(L, -1) + Um
    return info == 0 and np.array_equal(got, ref) and np.all(LU[1] == 0)


def pin_lu_pivoted_factors():
    """A = P L U with |l_ij| <= 3/8 and small integer U: partial pivoting
    must undo P, and with dyadic entries every operation is exact, so the
    stored factors are exactly L (strictly lower part, in the pivoted row
    order) and U, with zero low words.  This needs the row interchanges to
    carry the multipliers already stored left of the pivot column."""
    rng = np.random.default_rng(8)
    n = 6
    Lm = np.eye(n) + np.tril(rng.integers(-3, 4, (n, n)) / 8.0, -1)
    Um = np.triu(rng.integers(-9, 10, (n, n)).astype(float), 1) + \
        np.diag(rng.choice([-1, 1], n) * rng.integers(12, 20, n))
    A = np.zeros((2, n, n))
    A[0] = (Lm @ Um)[rng.permutation(n)].T
    LU, piv, info = oracle.lu(2, A)
    return info == 0 and np.array_equal(LU[0].T, np.tril(Lm, -1) + Um) and np.all(LU[1] == 0)


def pin_solve_exact():
    """A = P L U with |l_ij| <= 3/8, small integer U with a power-of-two
    diagonal, and an integer x*: every step of the substitution is exact
    (the reciprocals 1/u_jj included), so x = x* with zero low words."""
    rng = np.random.default_rng(9)
    n = 6
    Lm = np.eye(n) + np.tril(rng.integers(-3, 4, (n, n)) / 8.0, -1)
    Um = np.triu(rng.integers(-9, 10, (n, n)).astype(float), 1) + \
        np.diag(rng.choice([-16.0, -8.0, 8.0, 16.0], n))
    xs = rng.integers(-5, 6, n).astype(float)
    M = (Lm @ Um)[rng.permutation(n)]
    A = np.zeros((2, n, n)); A[0] = M.T
    b = np.zeros((2, n)); b[0] = M @ xs
    LU, piv, info = oracle.lu(2, A)
    x = oracle.solve(2, LU, piv, b)
    return info == 0 and np.array_equal(x[0], xs) and np.all(x[1] == 0)


def pin_residual():
    rng = np.random.default_rng(5)
    n = 5
    A = np.zeros((2, n, n)); A[0] = rng.uniform(-1, 1, (n, n)); A[1] = A[0] * 2.0 ** -60
    x = np.zeros((3, n)); x[0] = rng.uniform(-1, 1, n); x[1] = x[0] * 2.0 ** -70
    b = np.zeros((1, n)); b[0] = rng.uniform(-1, 1, n)
    r = oracle.residual(A, b, x, 8)
    rf = X.residual(X.mat_to_frac(A, n), X.vec_to_frac(b), X.vec_to_frac(x))
    return all(list(r[:, i]) == X.greedy_words(rf[i], 8) for i in range(n))


def pin_rn_ties():
    return oracle.exact_sum([1.0, 2.0 ** -53], 1)[0] == 1.0 and \
        oracle.exact_sum([1.0, 3 * 2.0 ** -53], 1)[0] == 1.0 + 2.0 ** -51


def pin_rn_sticky():
    """Above the halfway point by less than the last place's half: the bits
    below the rounding bit decide, so 1 + 2^-53 + 2^-80 rounds up to
    1 + 2^-52 (and its negative down), even though 1 is the even neighbour."""
    up = oracle.exact_sum([1.0, 2.0 ** -53, 2.0 ** -80], 1)[0]
    down = oracle.exact_sum([-1.0, -2.0 ** -53, -2.0 ** -80], 1)[0]
    return up == 1.0 + 2.0 ** -52 and down == -(1.0 + 2.0 ** -52)


def pin_solve_pivots():
    n = 5
    perm = [3, 0, 4, 1, 2]
    A = np.zeros((2, n, n))
    for i in range(n):
        A[0, perm[i], i] = 1.0
    LU, piv, _ = oracle.lu(2, A)
    b = np.zeros((2, n)); b[0] = np.arange(1.0, n + 1)
    x = oracle.solve(2, LU, piv, b)
    ref = np.zeros(n)
    for i in range(n):
        ref[perm[i]] = b[0, i]
    return np.array_equal(x[0], ref)


def pin_refine():
    s = W.svd_system(12, 8.0, seed=6)
    st, x, corr, nres, info = oracle.refine(s.A, s.b, 2)
    return st == 0 and X.forward_error(X.vec_to_frac(x), [Fraction(1)] * 12) <= Fraction(1, 2 ** 200)


def pin_back_substitution_reciprocal():
    """Reading of the back substitution (Section 2, Listing 1's SolveTDLSPM
    does not fix the order): d_j = 1/u_jj first, then x_j = y_j d_j.  For
    u = 35, y = 105 (DD, QD) and u = 45, y = 45 (TD) the quotient y/u is an
    integer, which a division returns exactly, while y times the rounded
    reciprocal misses it by a few units in the last place."""
    for w, u, y in ((2, 35, 105), (3, 45, 45), (4, 35, 105)):
        A = np.zeros((w, 1, 1)); A[0, 0, 0] = float(u)
        LU, piv, info = oracle.lu(w, A)
        b = np.zeros((w, 1)); b[0, 0] = float(y)
        x = X.words_to_frac(oracle.solve(w, LU, piv, b)[:, 0])
        k = Fraction(y, u)
        if x == k or abs(x - k) > 4 * U ** w * k:
            return False
    return True


def pin_stagnation_exit():
    """Stop mode 1's stagnation exit, traced by hand on a 1 x 1 system.
    A = 1 + 0 - 3/4 + 0 = 1/4 in four words, whose leading DD words give the
    inner factor 1; b = 1, so x* = 4.  x0 = 1.  Each step solves with 1
    instead of 1/4, so the error shrinks by 3/4 per correction:
    r0 = 3/4 -> correction 3/4 (x1 = 7/4);  r1 = 9/16 -> correction 9/16
    (x2 = 37/16).  The second correction exceeds half the first, so the
    loop stops there as not converged: status 2 after 2 corrections and 2
    residuals, with x = 37/16 exactly."""
    A = np.zeros((4, 1, 1)); A[0, 0, 0] = 1.0; A[2, 0, 0] = -0.75
    b = np.ones((1, 1))
    st, x, corr, nres, info = oracle.refine(A, b, 2)
    return (st, corr, nres, info) == (2, 2, 2, 0) and x[0, 0] == 37 / 16 and not np.any(x[1:, 0])


def _rel_bound(w, op):
    """The relative error bounds the arithmetic is held to: DD multiply 5u^2
    and divide 15u^2 (Joldes, Muller and Popescu 2017), TD/QD 4u^w."""
    if w == 2:
        return (5 if op == oracle.OP_MUL else 15) * U ** 2
    return 4 * U ** w


def pin_rel(op, w):
    def f():
        rng = np.random.default_rng(20 + w)
        x, y = _rand_mw(rng, w, 200), _rand_mw(rng, w, 200)
        z = oracle.arith(op, w, x, y)
        for i in range(200):
            a, b = X.words_to_frac(x[:, i]), X.words_to_frac(y[:, i])
            ex = a * b if op == oracle.OP_MUL else a / b
            if abs(X.words_to_frac(z[:, i]) - ex) > _rel_bound(w, op) * abs(ex):
                return False
        return True
    return f


def pin_cmpabs(w):
    """The pivot order on |x| against the exact order, with near ties in the
    last word, exact ties and random signs."""
    def f():
        rng = np.random.default_rng(30 + w)
        x = _rand_mw(rng, w, 400)
        y = x.copy()
        y[w - 1] += np.where(rng.random(400) < 0.5, 1, -1) * np.abs(x[w - 1]) * 2.0 ** -10
        flip = rng.random(400) < 0.5
        y[:, flip] = -y[:, flip]
        x[:, rng.random(400) < 0.5] *= -1
        y[:, ::7] = x[:, ::7]
        r = oracle.arith(oracle.OP_CMPABS, w, x, y)
        for i in range(400):
            a, b = abs(X.words_to_frac(x[:, i])), abs(X.words_to_frac(y[:, i]))
            if r[i] != (a > b) - (a < b):
                return False
        return True
    return f


def pin_singular_info():
    """A zero column at position 2 (0-based) of a 5 x 5 matrix: the first
    exactly zero pivot is at step 3 in the 1-based count that info uses
    (LAPACK getrf)."""
    rng = np.random.default_rng(7)
    A = np.zeros((2, 5, 5))
    A[0] = rng.uniform(-1, 1, (5, 5))
    A[:, 2, :] = 0.0
    _, _, info = oracle.lu(2, A)
    return info == 3


def pin_eq2_first_exit():
    """Stop mode 0 (Eq. (2)) stops at the first iterate that meets
    ||r||_2 <= sqrt(n) rtol ||A||_F ||x||_2.  rtol is placed so that after one
    correction ||r|| lies halfway (a factor 2 either side) between
    rtol ||A|| ||x|| and sqrt(n) rtol ||A|| ||x|| (n = 16), from exact
    residuals: the loop must stop after exactly one correction."""
    import math
    s = W.svd_system(16, 8.0, seed=4)
    n = 16
    _, x1, c1, _, _ = oracle.refine(s.A, s.b, 2, stop_mode=0, rtol=0.0, max_iter=1)
    Af = X.mat_to_frac(s.A, n)
    r = X.residual(Af, X.vec_to_frac(s.b), X.vec_to_frac(x1))
    nr2 = sum(v * v for v in r)
    nA2 = sum(a * a for row in Af for a in row)
    nx2 = sum(v * v for v in X.vec_to_frac(x1))
    ratio = math.sqrt(float(nr2 / (nA2 * nx2)))
    st, x, corr, nres, info = oracle.refine(s.A, s.b, 2, stop_mode=0, rtol=ratio / 2)
    return c1 == 1 and st == 0 and corr == 1


MUTATIONS = [
    ("dd_mul drops the cross terms", "    cl3 = cl1 + cl2;\n", "    cl3 = cl1;\n", pin_dd_mul),
    ("dd_add wrong sign", "    c = sl + th;\n", "    c = sl - th;\n", pin_add(2)),
    ("renorm drops the cascade errors", "        t[i + 1] = lo;\n", "        t[i + 1] = 0.0;\n", pin_add(3)),
    ("quad-word add drops a word", "        t[m++] = e[i - 1];\n", "        t[m++] = 0.0 * e[i - 1];\n", pin_add(4)),
    ("TwoProd error term lost", "    *e = fma(a, b, -pp);\n", "    *e = 0.0 * fma(a, b, -pp);\n", pin_twoprod),
    ("pivot ties take the last row", "if (mw_cmpabs(w, v, best) > 0) {", "if (mw_cmpabs(w, v, best) >= 0) {", pin_lu_ties),
    ("LU update adds instead of subtracting", "                mw_sub(w, a, prod, res);\n                st_m(w, A, plane, j * lda + ii, res);",
     "                mw_add(w, a, prod, res);\n                st_m(w, A, plane, j * lda + ii, res);", pin_lu_factors),
    ("residual sign flipped", "acc_add_prod(a, aij, x[d * n + j], 1, 0);", "acc_add_prod(a, aij, x[d * n + j], 0, 0);", pin_residual),
    ("rounding ties away from even", "(acc_any_below(a, lsb - 1) || (q & 1u))", "(acc_any_below(a, lsb - 1) || 1)", pin_rn_ties),
    ("solve ignores the pivots", "        int64_t p = piv[k];\n        if (p != k) {", "        int64_t p = piv[k];\n        if (0 && p != k) {", pin_solve_pivots),
    ("refinement forgets to scale back", "acc_add_double(&a, z[c * n + i], er);", "acc_add_double(&a, z[c * n + i], 0);", pin_refine),
    ("back substitution divides by u_jj", "        mw_mul(w, yj, dj, xj);\n",
     "        { double uu[4]; ld_m(w, LU, plane, j * lda + j, uu); mw_div(w, yj, uu, xj); }\n",
     pin_back_substitution_reciprocal),
    ("stagnation test against twice the previous correction", "corr > 0.5 * prev", "corr > 2.0 * prev",
     pin_stagnation_exit),
    ("stagnation test never updates the previous correction", "            prev = corr;\n", "\n",
     pin_stagnation_exit),
    ("stagnation test starts a correction late", "if (corrections >= 2 && corr > 0.5 * prev)",
     "if (corrections >= 3 && corr > 0.5 * prev)", pin_stagnation_exit),
    ("DD division drops its correction quotient", "    fast_two_sum(q0, q1, &z[0], &z[1]);\n",
     "    fast_two_sum(q0, 0.0 * q1, &z[0], &z[1]);\n", pin_rel(oracle.OP_DIV, 2)),
    ("DD division ignores the divisor's low word", "    pl = fma(y[1], q0, pl);", "    pl = fma(0.0 * y[1], q0, pl);",
     pin_rel(oracle.OP_DIV, 2)),
    ("TD multiplication drops x1*y1", "        c = x[1] * y[1];\n", "        c = 0.0 * x[1] * y[1];\n",
     pin_rel(oracle.OP_MUL, 3)),
    ("QD multiplication drops an order-2 product error", "        c = c + q11;\n", "        c = c + 0.0 * q11;\n",
     pin_rel(oracle.OP_MUL, 4)),
    ("long division's remainder loses the product errors", "        t[m++] = q[i - 1];\n",
     "        t[m++] = 0.0 * q[i - 1];\n", pin_rel(oracle.OP_DIV, 3)),
    ("magnitude order without the sign adjustment", "        double a = sx * x[c], b = sy * y[c];\n",
     "        double a = x[c], b = y[c];\n", pin_cmpabs(2)),
    ("zero pivot reported 0-based", "            if (*info == 0) *info = k + 1;\n",
     "            if (*info == 0) *info = k;\n", pin_singular_info),
    ("Eq. (2) without its sqrt(n) factor", "            double rhs = sqrt((double)n) * rtol;\n",
     "            double rhs = rtol;\n", pin_eq2_first_exit),
    ("Eq. (2) without the norm of x", "            rhs = rhs * nx;\n", "            rhs = rhs * 1.0;\n",
     pin_eq2_first_exit),
    ("row interchange skips the multipliers left of the pivot",
     "        if (p != k) {\n            for (j = 0; j < n; ++j) {\n",
     "        if (p != k) {\n            for (j = k; j < n; ++j) {\n", pin_lu_pivoted_factors),
    ("forward substitution also updates the diagonal row",
     "        for (i = j + 1; i < n; ++i) {\n            double l[4], yi[4], prod[4], res[4];\n",
     "        for (i = j; i < n; ++i) {\n            double l[4], yi[4], prod[4], res[4];\n", pin_solve_exact),
    ("back substitution skips row 0",
     "        for (i = 0; i < j; ++i) {\n            double u[4], yi[4], prod[4], res[4];\n",
     "        for (i = 1; i < j; ++i) {\n            double u[4], yi[4], prod[4], res[4];\n", pin_solve_exact),
    ("greedy rounding keeps the rounded word in the accumulator",
     "        acc_add_u128(a, 1, (unsigned __int128)q, lsb);\n",
     "        acc_add_u128(a, 1, (unsigned __int128)0, lsb);\n", pin_residual),
    ("carries taken with an unsigned shift",
     "        int64_t c = a->d[k] >> 32;  /* arithmetic shift = floor division */\n",
     "        int64_t c = (int64_t)((uint64_t)a->d[k] >> 32);\n", pin_residual),
    ("rounding ignores the sticky bits", "(acc_any_below(a, lsb - 1) || (q & 1u))", "((q & 1u))", pin_rn_sticky),
    ("TwoSum drops the error of b", "    *e = da + db;\n", "    *e = da;\n", pin_twosum),
    ("FastTwoSum error with the wrong sign", "    *e = b - z;\n", "    *e = z - b;\n", pin_fasttwosum),
]


@pytest.mark.parametrize("name,old,new,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(name, old, new, pin, tmp_path):
    assert pin(), "the pin must pass on the unmodified oracle"
    src = oracle.source_text()
    assert src.count(old) == 1, "mutation anchor must be unique"
    path = oracle.compile_variant(src.replace(old, new), str(tmp_path / "libmwo_mut.so"))
    with oracle.use(path):
        caught = not pin()
    assert caught, name
