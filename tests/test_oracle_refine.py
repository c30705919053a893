"""Pins for the oracle's mixed precision iterative refinement (Section 2,
Listing 1; stopping test Eq. (2)): exact known solutions, exact rational
solutions, Cramer solutions, edge cases, and the shape of Tables 1-2 on the
paper's own problem (Section 3, Eq. (1)) at a reduced n."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import exact as X
from paper_2107_12550_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")
TWO_M200 = Fraction(1, 2 ** 200)


def _fe(x, xs):
    return X.forward_error(X.vec_to_frac(x), xs)


@pytest.mark.parametrize("w_in", [2, 3, 4])
def test_refine_svd_known_solution(w_in):
    """A = U diag(sigma) V^T, kappa = 2^33, b = A * ones exactly (8 words):
    the refined x must equal ones to 2^-200."""
    s = W.svd_system(24, 10.0, seed=3)
    st, x, corr, nres, info = oracle.refine(s.A, s.b, w_in)
    assert st == 0 and info == 0
    assert 1 <= corr <= 6
    assert _fe(x, [Fraction(1)] * 24) <= TWO_M200


def test_refine_exact_rational_solution_of_dd_rhs():
    """b rounded to DD: x* is the exact rational solution of the stored
    system (not ones); the refined x must match it to 2^-200."""
    s = W.uniform_system(12, words=2, seed=9, b_words=2)
    xs = X.solve(X.mat_to_frac(s.A, 12), X.vec_to_frac(s.b))
    st, x, corr, nres, info = oracle.refine(s.A, s.b, 2, target_bits=200)
    assert st == 0
    assert _fe(x, xs) <= TWO_M200
    assert xs != [Fraction(1)] * 12


def test_refine_integer_system_cramer():
    rng = np.random.default_rng(77)
    n = 6
    Mi = [[int(rng.integers(-9, 10)) for _ in range(n)] for _ in range(n)]
    bi = [int(rng.integers(-9, 10)) for _ in range(n)]
    xs = X.cramer_solve_int(Mi, bi)
    A = np.zeros((1, n, n))
    for i in range(n):
        for j in range(n):
            A[0, j, i] = Mi[i][j]
    b = np.zeros((1, n)); b[0] = bi
    for w_in in (2, 3):
        st, x, corr, nres, info = oracle.refine(A, b, w_in, target_bits=300)
        assert st == 0
        assert _fe(x, xs) <= Fraction(1, 2 ** 300)


def test_refine_edge_cases():
    s = W.svd_system(10, 6.0, seed=1)
    st, x, corr, nres, info = oracle.refine(s.A, s.b, 2, max_iter=0)
    assert st == 2 and corr == 0 and nres == 1
    # zero matrix: singular LU
    Z = np.zeros((2, 4, 4))
    st, x, corr, nres, info = oracle.refine(Z, np.ones((2, 4)), 2)
    assert st == 1 and info == 1
    # n = 1
    A = np.array([[[3.0]]])
    b = np.array([[1.0]])
    st, x, corr, nres, info = oracle.refine(A, b, 2, target_bits=400)
    assert st == 0
    assert abs(X.words_to_frac(x[:, 0]) - Fraction(1, 3)) <= Fraction(1, 3) * Fraction(1, 2 ** 400)


def test_refine_eq2_stopping_rule_meets_its_bound():
    """stop_mode 0 (Eq. (2)): on exit ||r||_2 <= sqrt(n) rtol ||A||_F ||x||_2."""
    s = W.svd_system(16, 8.0, seed=4)
    rtol = 1e-60
    st, x, corr, nres, info = oracle.refine(s.A, s.b, 2, stop_mode=0, rtol=rtol)
    assert st == 0
    n = 16
    Af = X.mat_to_frac(s.A, n)
    r = X.residual(Af, X.vec_to_frac(s.b), X.vec_to_frac(x))
    nr2 = sum(v * v for v in r)
    nA2 = sum(a * a for row in Af for a in row)
    nx2 = sum(v * v for v in X.vec_to_frac(x))
    # squared form of Eq. (2), with a 1% allowance for the leading-word norms
    assert float(nr2) <= (1.01 * n ** 0.5 * rtol) ** 2 * float(nA2) * float(nx2)


def test_paper_problem_shape_matches_tables():
    """The paper's problem (Eq. (1)) at n = 96 instead of 2000: the direct
    solutions' errors fall by many orders from DD to TD to QD (Table 1:
    1e-1, 1e-17, 1e-34), refinement with the 424-bit residual and Eq. (2)
    at 10^-100 reaches Max.RE <= 1e-70 for every inner precision (Table 2:
    1e-77 .. 1e-98), and the iteration counts order DD > TD >= QD >= 1 with
    QD at one or two iterations (Table 2: 15, 2, 1)."""
    with open(GOLDEN) as f:
        g = json.load(f)
    n = 96
    s = W.paper_system(n, seed=2)
    xs = [Fraction(int(v)) for v in s.x_star]

    def maxre(x):
        xf = X.vec_to_frac(x)
        return max(abs(xf[i] - xs[i]) / xs[i] for i in range(1, n))

    direct = {}
    iters = {}
    for w, name in ((2, "DD"), (3, "TD"), (4, "QD")):
        LU, piv, info = oracle.lu(w, s.A)
        direct[name] = maxre(oracle.solve(w, LU, piv, s.b))
        st, x, corr, nres, _ = oracle.refine(s.A, s.b, w, stop_mode=0, rtol=1e-100, max_iter=40)
        assert st == 0
        iters[name] = corr
        assert maxre(x) <= Fraction(1, 10 ** 70)
    t1 = g["table1_max_rel_err"]
    assert direct["DD"] > direct["TD"] * Fraction(10 ** 10) > 0
    assert direct["TD"] > direct["QD"] * Fraction(10 ** 10)
    # same order of magnitude as Table 1 within the n-dependence (<= 1e6)
    for name in ("TD", "QD"):
        assert float(direct[name]) <= 1e6 * t1[name]
    assert iters["DD"] > iters["TD"] >= iters["QD"] >= 1
    assert iters["QD"] <= 2 and iters["TD"] <= 4
    assert iters["DD"] <= 2 * max(g["table2"]["DD"]["iters"])
