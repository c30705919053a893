"""Exact rational arithmetic (``fractions.Fraction``) used to pin the C oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Everything here is
exact: binary64 words become dyadic rationals, Gaussian elimination runs on
rationals, and rounding back to words is the greedy round-to-nearest
c_i = RN(x - sum_{j<i} c_j) (CPython's int/int true division, used by
``float(Fraction)``, is correctly rounded, ties to even).
"""
from __future__ import annotations

from fractions import Fraction
from typing import List, Sequence

import numpy as np


def frac(v: float) -> Fraction:
    return Fraction(float(v))


def words_to_frac(words: Sequence[float]) -> Fraction:
    """Exact value of a multiword number (sum of its words)."""
    return sum((Fraction(float(w)) for w in words), Fraction(0))


def vec_to_frac(v: np.ndarray) -> List[Fraction]:
    """(w, n) array -> list of n exact values."""
    return [words_to_frac(v[:, i]) for i in range(v.shape[1])]


def mat_to_frac(A: np.ndarray, n: int | None = None) -> List[List[Fraction]]:
    """(w, n, lda) array -> row-major list of lists of exact values."""
    if n is None:
        n = A.shape[1]
    return [[words_to_frac(A[:, j, i]) for j in range(n)] for i in range(n)]


def greedy_words(x: Fraction, nw: int) -> List[float]:
    """Greedy round-to-nearest expansion of x into nw binary64 words."""
    out = []
    r = x
    for _ in range(nw):
        c = float(r)
        out.append(c)
        r -= Fraction(c)
    return out


def cmpabs_exact(a: Fraction, b: Fraction) -> int:
    return (abs(a) > abs(b)) - (abs(a) < abs(b))


def lu_pp(A: List[List[Fraction]]):
    """Exact LU with partial pivoting (first index on ties).
    Returns (L\\U as a list of lists, piv list, info)."""
    n = len(A)
    M = [row[:] for row in A]
    piv = []
    info = 0
    for k in range(n):
        p = k
        for i in range(k + 1, n):
            if abs(M[i][k]) > abs(M[p][k]):
                p = i
        piv.append(p)
        if p != k:
            M[k], M[p] = M[p], M[k]
        if M[k][k] == 0:
            if info == 0:
                info = k + 1
            continue
        for i in range(k + 1, n):
            M[i][k] = M[i][k] / M[k][k]
        for i in range(k + 1, n):
            lik = M[i][k]
            if lik == 0:
                continue
            for j in range(k + 1, n):
                M[i][j] -= lik * M[k][j]
    return M, piv, info


def solve(A: List[List[Fraction]], b: List[Fraction]) -> List[Fraction]:
    """Exact solution of A x = b (A nonsingular)."""
    n = len(A)
    M, piv, info = lu_pp(A)
    if info:
        raise ZeroDivisionError("singular matrix")
    y = list(b)
    for k in range(n):
        p = piv[k]
        if p != k:
            y[k], y[p] = y[p], y[k]
    for j in range(n):
        for i in range(j + 1, n):
            y[i] -= M[i][j] * y[j]
    for j in range(n - 1, -1, -1):
        y[j] = y[j] / M[j][j]
        for i in range(j):
            y[i] -= M[i][j] * y[j]
    return y


def matvec(A: List[List[Fraction]], x: List[Fraction]) -> List[Fraction]:
    return [sum((a * xi for a, xi in zip(row, x)), Fraction(0)) for row in A]


def residual(A: List[List[Fraction]], b: List[Fraction], x: List[Fraction]):
    Ax = matvec(A, x)
    return [bi - axi for bi, axi in zip(b, Ax)]


def inf_norm_vec(v: Sequence[Fraction]) -> Fraction:
    return max((abs(t) for t in v), default=Fraction(0))


def inf_norm_mat(A: List[List[Fraction]]) -> Fraction:
    return max((sum((abs(a) for a in row), Fraction(0)) for row in A), default=Fraction(0))


def backward_error(A, b, x) -> Fraction:
    """Normwise backward error ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)."""
    r = residual(A, b, x)
    den = inf_norm_mat(A) * inf_norm_vec(x) + inf_norm_vec(b)
    return inf_norm_vec(r) / den if den else Fraction(0)


def forward_error(x, xstar) -> Fraction:
    """||x - x*||_inf / ||x*||_inf."""
    d = inf_norm_vec([a - b for a, b in zip(x, xstar)])
    s = inf_norm_vec(xstar)
    return d / s if s else d


def det_bareiss(A: List[List[int]]) -> int:
    """Exact determinant of an integer matrix by Bareiss' fraction-free
    elimination (with row swaps)."""
    n = len(A)
    M = [row[:] for row in A]
    sign = 1
    prev = 1
    for k in range(n - 1):
        if M[k][k] == 0:
            for i in range(k + 1, n):
                if M[i][k] != 0:
                    M[k], M[i] = M[i], M[k]
                    sign = -sign
                    break
            else:
                return 0
        for i in range(k + 1, n):
            for j in range(k + 1, n):
                M[i][j] = (M[i][j] * M[k][k] - M[i][k] * M[k][j]) // prev
        prev = M[k][k]
    return sign * M[n - 1][n - 1]


def cramer_solve_int(A: List[List[int]], b: List[int]) -> List[Fraction]:
    """Exact solution of an integer system by Cramer's rule with Bareiss
    determinants (independent of the elimination in ``solve``)."""
    n = len(A)
    d = det_bareiss(A)
    if d == 0:
        raise ZeroDivisionError("singular matrix")
    x = []
    for j in range(n):
        Aj = [row[:j] + [b[i]] + row[j + 1:] for i, row in enumerate(A)]
        x.append(Fraction(det_bareiss(Aj), d))
    return x
