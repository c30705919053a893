"""Planted mistakes: each test compiles a copy of the oracle with one
plausible error (a dropped term, a wrong sign, a wrong index or tie rule)
and shows that a pin rejects it, while the unmodified oracle passes the
same pin.  Mistakes are planted in the oracle only, on the CPU."""
import os
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
