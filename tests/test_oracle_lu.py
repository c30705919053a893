"""Pins for the oracle's LU with partial pivoting and substitution (the
direct method of the paper: Section 2, Listing 1, TDLUdecompPM and
SolveTDLSPM), checked against exact rational Gaussian elimination, exactly
factorable matrices, permutations, singular cases and an independent Cramer
(Bareiss) solve."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import exact as X
from paper_2107_12550_gb300 import workloads as W

U = Fraction(1, 2 ** 53)


def _planar(M, w, lda=None):
    """Row-major list of doubles -> (w, n, lda) with word 0 = M."""
    n = len(M)
    lda = lda or n + 1
    A = np.zeros((w, n, lda))
    for i in range(n):
        for j in range(n):
            A[0, j, i] = float(M[i][j])
    return A


def _apply_swaps_rows(M, piv):
    M = [row[:] for row in M]
    for k, p in enumerate(piv):
        if p != k:
            M[k], M[p] = M[p], M[k]
    return M


def _factorable(n, rng, zero_diag_at=None):
    """A with P A = L U exactly: L unit lower with entries k/8, |k| < 8 (so
    |l| < 1 and pivots are unique), U upper with small integers; A is formed
    by undoing a random swap sequence.  All values are small dyadics, so
    every multiword operation on them is exact."""
    piv = [int(rng.integers(k, n)) for k in range(n)]
    L = [[Fraction(0)] * n for _ in range(n)]
    Um = [[Fraction(0)] * n for _ in range(n)]
    for i in range(n):
        L[i][i] = Fraction(1)
        for j in range(i):
            L[i][j] = Fraction(int(rng.integers(-7, 8)), 8)
        for j in range(i, n):
            Um[i][j] = Fraction(int(rng.integers(-9, 10)))
        if Um[i][i] == 0:
            Um[i][i] = Fraction(5)
    if zero_diag_at is not None:
        Um[zero_diag_at][zero_diag_at] = Fraction(0)
    M = [[sum((L[i][k] * Um[k][j] for k in range(n)), Fraction(0)) for j in range(n)]
         for i in range(n)]
    A = [row[:] for row in M]
    for k in range(n - 1, -1, -1):          # A = P^-1 M
        p = piv[k]
        if p != k:
            A[k], A[p] = A[p], A[k]
    return A, L, Um, piv


@pytest.mark.parametrize("w", [2, 3, 4])
def test_lu_recovers_exact_factors(w):
    rng = np.random.default_rng(100 + w)
    for n in (1, 2, 5, 9, 16):
        A, L, Um, piv = _factorable(n, rng)
        LU, p, info = oracle.lu(w, _planar(A, w))
        assert info == 0
        assert list(p) == piv
        for i in range(n):
            for j in range(n):
                ref = L[i][j] if i > j else Um[i][j]
                assert X.words_to_frac(LU[:, j, i]) == ref, (n, i, j)


@pytest.mark.parametrize("w", [2, 3, 4])
def test_lu_singular_info(w):
    rng = np.random.default_rng(110 + w)
    A, L, Um, piv = _factorable(7, rng, zero_diag_at=3)
    # entries below the zero pivot are zero too, so the pivot search finds 0
    LU, p, info = oracle.lu(w, _planar(A, w))
    assert info == 4
    Z = _planar([[0.0] * 3 for _ in range(3)], w)
    _, _, info0 = oracle.lu(w, Z)
    assert info0 == 1


@pytest.mark.parametrize("w", [2, 3, 4])
def test_lu_permutation_matrix(w):
    rng = np.random.default_rng(120 + w)
    n = 11
    perm = rng.permutation(n)
    P = [[1.0 if perm[i] == j else 0.0 for j in range(n)] for i in range(n)]
    LU, piv, info = oracle.lu(w, _planar(P, w))
    assert info == 0
    assert _apply_swaps_rows(P, piv) == [[1.0 if i == j else 0.0 for j in range(n)] for i in range(n)]
    for i in range(n):
        for j in range(n):
            assert LU[0, j, i] == (1.0 if i == j else 0.0)
            assert np.all(LU[1:, j, i] == 0)


@pytest.mark.parametrize("w", [2, 3, 4])
def test_lu_ties_take_first_row(w):
    """Equal magnitudes in the pivot column: the first row wins (LAPACK)."""
    M = [[1.0, 2.0, 3.0], [-1.0, 5.0, 1.0], [1.0, 1.0, 7.0]]
    _, piv, info = oracle.lu(w, _planar(M, w))
    assert piv[0] == 0 and info == 0
    M = [[0.5, 2.0, 3.0], [-1.0, 5.0, 1.0], [1.0, 1.0, 7.0]]
    _, piv, _ = oracle.lu(w, _planar(M, w))
    assert piv[0] == 1


@pytest.mark.parametrize("w", [2, 3, 4])
def test_lu_matches_exact_pivoting_and_backward_error(w):
    """On random matrices the pivots equal those of exact elimination and
    the factor error ||P A - L U||_inf <= 4 n u^w ||A||_inf."""
    for n in (3, 8, 13):
        A = W.uniform_matrix(n, w, seed=7 * n + w, lda=n + 2)
        LU, piv, info = oracle.lu(w, A)
        Af = X.mat_to_frac(A, n)
        _, piv_exact, _ = X.lu_pp(Af)
        assert list(piv) == piv_exact
        PA = _apply_swaps_rows(Af, list(piv))
        Lf = [[X.words_to_frac(LU[:, j, i]) if i > j else (Fraction(1) if i == j else Fraction(0))
               for j in range(n)] for i in range(n)]
        Uf = [[X.words_to_frac(LU[:, j, i]) if i <= j else Fraction(0) for j in range(n)]
              for i in range(n)]
        E = [[PA[i][j] - sum((Lf[i][k] * Uf[k][j] for k in range(n)), Fraction(0))
              for j in range(n)] for i in range(n)]
        assert X.inf_norm_mat(E) <= 4 * n * U ** w * X.inf_norm_mat(Af)


@pytest.mark.parametrize("w", [2, 3, 4])
def test_solve_backward_error_and_known_solution(w):
    for n in (1, 6, 17):
        A = W.uniform_matrix(n, w, seed=31 * n + w, lda=n + 1)
        b = W.rowsum_words(A, None, w)
        LU, piv, info = oracle.lu(w, A)
        x = oracle.solve(w, LU, piv, b)
        Af = X.mat_to_frac(A, n)
        bf = X.vec_to_frac(b)
        xf = X.vec_to_frac(x)
        eta = X.backward_error(Af, bf, xf)
        assert eta <= 4 * n * U ** w, float(eta)
        xs = X.solve(Af, bf)
        # forward error within the condition-number bound (kappa from exact inverse rows)
        fe = X.forward_error(xf, xs)
        assert fe <= Fraction(1, 10 ** 10) * 10 ** (-(16 * (w - 2)))


def test_solve_integer_system_cramer():
    """An integer system solved exactly by Cramer's rule (Bareiss
    determinants, independent of elimination)."""
    rng = np.random.default_rng(5)
    n = 7
    Mi = [[int(rng.integers(-20, 21)) for _ in range(n)] for _ in range(n)]
    bi = [int(rng.integers(-50, 51)) for _ in range(n)]
    xs = X.cramer_solve_int(Mi, bi)
    assert X.matvec([[Fraction(v) for v in r] for r in Mi], xs) == [Fraction(v) for v in bi]
    for w in (2, 3, 4):
        A = _planar(Mi, w)
        b = np.zeros((w, n)); b[0] = bi
        LU, piv, info = oracle.lu(w, A)
        x = oracle.solve(w, LU, piv, b)
        fe = X.forward_error(X.vec_to_frac(x), xs)
        assert fe <= 1e4 * n * U ** w


def test_solve_applies_pivots_and_aliases():
    """b permuted consistently: solving P^T-scrambled identity systems."""
    n = 5
    perm = [3, 0, 4, 1, 2]
    P = [[1.0 if perm[i] == j else 0.0 for j in range(n)] for i in range(n)]
    for w in (2, 3, 4):
        LU, piv, _ = oracle.lu(w, _planar(P, w))
        b = np.zeros((w, n)); b[0] = np.arange(1.0, n + 1)
        x = oracle.solve(w, LU, piv, b)
        # P x = b  => x_j = b_i where perm[i] = j
        ref = np.zeros(n)
        for i in range(n):
            ref[perm[i]] = b[0, i]
        assert np.array_equal(x[0], ref)
