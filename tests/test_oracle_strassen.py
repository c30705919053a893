"""Pins of the oracle's block matrix product and its Strassen form
(Section 2: BNCmatmul and its Strassen variant) against exact results."""
import os
import types
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import exact as X
from oracle import strassen as S


def _int_mat(w, n, seed, lo=-8, hi=9):
    g = np.random.default_rng(seed)
    M = np.zeros((w, n, n))
    M[0] = g.integers(lo, hi, (n, n)).astype(float)
    return M


@pytest.mark.parametrize("levels", [0, 1, 2, 3])
@pytest.mark.parametrize("w", [2, 3, 4])
def test_exact_on_small_integers(w, levels):
    """Small integer entries keep every intermediate exact, so both forms
    equal the integer product exactly: this pins the quadrant bookkeeping
    and the signs of all seven products and eighteen additions."""
    n = 16
    A = _int_mat(w, n, 10 + levels)
    B = _int_mat(w, n, 20 + levels)
    ref = (A[0].T.astype(np.int64) @ B[0].T.astype(np.int64)).T        # (cols, rows) layout
    C = S.strassen(w, A, B, levels)
    assert np.array_equal(C[0], ref.astype(float))
    assert not C[1:].any()


def _mw_mat(w, n, seed):
    g = np.random.default_rng(seed)
    M = np.zeros((w, n, n))
    M[0] = g.uniform(-1, 1, (n, n))
    for c in range(1, w):
        _, ex = np.frexp(M[c - 1])
        M[c] = np.ldexp(g.uniform(-1, 1, (n, n)), ex - 54)
    return M


# error bounds per result relative to max|a| max|b|: the product ~ n u_w,
# Strassen ~ [(n/n0)^log2(12) (n0^2 + 5 n0) - 5n] u_w (Higham, Accuracy and
# Stability of Numerical Algorithms, Thm. 23.3), with slack
_LOG2_U = {2: -100, 3: -150, 4: -200}


@pytest.mark.parametrize("w", [2, 3, 4])
def test_error_bounds_against_exact_products(w):
    n = 32
    A = _mw_mat(w, n, 31 + w)
    B = _mw_mat(w, n, 41 + w)
    amax = np.max(np.abs(A[0]))
    bmax = np.max(np.abs(B[0]))
    for levels in (0, 1, 2):
        C = S.strassen(w, A, B, levels)
        n0 = n >> levels
        growth = n if levels == 0 else (n / n0) ** np.log2(12) * (n0 ** 2 + 5 * n0) - 5 * n
        bound = Fraction(growth) * Fraction(2) ** _LOG2_U[w] * Fraction(amax) * Fraction(bmax)
        worst = Fraction(0)
        for i in range(0, n, 3):
            for j in range(0, n, 5):
                ex = sum((X.words_to_frac(A[:, t, i]) * X.words_to_frac(B[:, j, t]) for t in range(n)), Fraction(0))
                worst = max(worst, abs(X.words_to_frac(C[:, j, i]) - ex))
        assert worst <= bound, (levels, float(worst), float(bound))
        if levels == 0:
            # the classical product is far inside its bound; a Strassen level
            # may lose more, but not orders of magnitude
            base_err = worst
    assert base_err > 0


def test_product_accumulates_from_c0():
    """product(w, A, B, C0) adds to C0 in ascending t (checked against the
    oracle's element-wise operations one step at a time)."""
    w, m, K, N = 3, 5, 4, 6
    g = np.random.default_rng(5)
    A = _mw_mat(w, 8, 1)[:, :K, :m].copy()
    B = _mw_mat(w, 8, 2)[:, :N, :K].copy()
    C0 = np.zeros((w, N, m))
    C0[0] = g.uniform(-1, 1, (N, m))
    got = S.product(w, A, B, C0)
    for j in range(N):
        for i in range(m):
            c = C0[:, j, i][:, None]
            for t in range(K):
                p = oracle.arith(oracle.OP_MUL, w, A[:, t, i][:, None], B[:, j, t][:, None])
                c = oracle.arith(oracle.OP_ADD, w, c, p)
            assert np.array_equal(got[:, j, i], c[:, 0])


def _strassen_variant(old: str, new: str):
    """A copy of the Strassen oracle with one planted mistake, loaded as a
    module of the oracle package."""
    path = os.path.join(os.path.dirname(S.__file__), "strassen.py")
    src = open(path).read()
    assert src.count(old) == 1, old
    mod = types.ModuleType("oracle.strassen_variant")
    mod.__package__ = "oracle"
    exec(compile(src.replace(old, new), path + " (variant)", "exec"), mod.__dict__)
    return mod


def _exact_one_level(model):
    n = 8
    A = _int_mat(2, n, 51)
    B = _int_mat(2, n, 52)
    ref = (A[0].T.astype(np.int64) @ B[0].T.astype(np.int64)).T
    return np.array_equal(model.strassen(2, A, B, 1)[0], ref.astype(float))


STRASSEN_MUTATIONS = [
    ("C12 and C21 written to each other's quadrant",
     "    C[:, h:n, 0:h] = add(M3, M5)                        # C12 (block row 0, block column 1)\n"
     "    C[:, 0:h, h:n] = add(M2, M4)                        # C21\n",
     "    C[:, 0:h, h:n] = add(M3, M5)\n    C[:, h:n, 0:h] = add(M2, M4)\n"),
    ("M6 with its difference reversed", "    M6 = rec(sub(A21, A11), add(B11, B12))\n",
     "    M6 = rec(sub(A11, A21), add(B11, B12))\n"),
    ("C11 without M7", "    C[:, 0:h, 0:h] = add(sub(add(M1, M4), M5), M7)      # C11\n",
     "    C[:, 0:h, 0:h] = sub(add(M1, M4), M5)\n"),
]


@pytest.mark.parametrize("name,old,new", STRASSEN_MUTATIONS, ids=[m[0] for m in STRASSEN_MUTATIONS])
def test_planted_strassen_mistake_is_caught(name, old, new):
    assert _exact_one_level(S), "the pin must pass on the unmodified oracle"
    assert not _exact_one_level(_strassen_variant(old, new)), name
