"""Pins of the split-product oracle (oracle/ozaki.py) against what the
mathematics fixes, independent of any implementation of the method:

* exactness: on entries with few significant bits every digit pair that
  matters is kept, so the slab product equals the exact product L U and
  the result equals the greedy DD rounding of C -/+ L U;
* the a-priori error bound of the truncated expansion,
  |P - L U|_ij <= 2^-107 max_t |l_it| max_t |u_tj|, on random DD data
  (the derivation: two floors per entry give |dx| < 2^(e - 119), hence
  2^(e_i + f_j - 113) over 64 terms; the dropped pairs p + q >= 17 add
  less than 2^(e_i + f_j - 112.1); and 2^(e_i + f_j) <= 16 max|l| max|u|);
* the digit expansion recomposes X exactly within the balanced ranges;
* C off the product's grid takes the rounded-product form, which then
  equals the DD subtraction of the greedily rounded product.
Planted mistakes in the model (a dropped diagonal, unbalanced digits) are
shown to fail these pins."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import exact as X
from oracle import ozaki as Z


def _dd_random(g, rows, cols, scale_rows=False):
    M = np.zeros((2, cols, rows))
    M[0] = g.uniform(-1, 1, (cols, rows))
    if scale_rows:
        M[0] *= np.ldexp(1.0, g.integers(-20, 20, rows))[None, :]
    _, ex = np.frexp(M[0])
    M[1] = np.where(M[0] == 0, 0.0, np.ldexp(g.uniform(-1, 1, (cols, rows)), ex - 55))
    return M


def _exact_prod(L, U, i, j, K):
    return sum((X.words_to_frac(L[:, t, i]) * X.words_to_frac(U[:, j, t]) for t in range(K)), Fraction(0))


def test_digits_recompose_within_ranges():
    g = np.random.default_rng(1)
    for _ in range(3000):
        x = int(g.integers(-2 ** 62, 2 ** 62)) * (1 << int(g.integers(0, 56)))
        a = Z.digits(x)
        assert sum(d * 256 ** (14 - p) for p, d in enumerate(a)) == x
        assert all(-128 <= d <= 127 for d in a[1:])
        if abs(x) < 2 ** 119:
            assert -128 <= a[0] <= 128


def test_small_integer_entries_are_exact():
    g = np.random.default_rng(2)
    m, N, K = 9, 7, 64
    L = np.zeros((2, K, m)); L[0] = g.integers(-100, 101, (K, m))
    U = np.zeros((2, N, K)); U[0] = g.integers(-100, 101, (N, K))
    C = np.zeros((2, N, m)); C[0] = g.integers(-10 ** 6, 10 ** 6, (N, m)) * 0.5
    for plus in (False, True):
        out, nexact = Z.update(C, L, U, m, N, K, plus=plus)
        assert nexact == m * N
        for i in range(m):
            for j in range(N):
                v = X.words_to_frac(C[:, j, i]) + (1 if plus else -1) * _exact_prod(L, U, i, j, K)
                assert list(out[:, j, i]) == X.greedy_words(v, 2)


def _worst_bound_ratio(model):
    g = np.random.default_rng(3)
    m, N, K = 12, 10, 64
    L = _dd_random(g, m, K, scale_rows=True)
    U = _dd_random(g, K, N)
    R, e, f = model(L, U, m, N, K)
    worst = Fraction(0)
    for i in range(m):
        for j in range(N):
            P = R[i][j] * Fraction(2) ** (e[i] + f[j] - 128)
            err = abs(P - _exact_prod(L, U, i, j, K))
            lim = Fraction(max(abs(L[0, :, i]))) * Fraction(max(abs(U[0, j, :])))
            worst = max(worst, err / lim)
    return worst


def test_truncated_expansion_error_bound():
    worst = _worst_bound_ratio(Z.slab_product)
    print(f"split slab product: max |P - LU| / (max|l| max|u|) = 2^{math.log2(worst):.1f}")
    assert worst <= Fraction(1, 2 ** 107)


def test_off_grid_c_takes_the_rounded_product_form():
    g = np.random.default_rng(4)
    m, N, K = 5, 4, 64
    L = _dd_random(g, m, K)
    U = _dd_random(g, K, N)
    C = np.zeros((2, N, m))
    C[0] = 2.0 ** -300 * g.uniform(1, 2, (N, m))     # far below the product's grid
    out, nexact = Z.update(C, L, U, m, N, K)
    assert nexact == 0
    R, e, f = Z.slab_product(L, U, m, N, K)
    for i in range(m):
        for j in range(N):
            P = R[i][j] * Fraction(2) ** (e[i] + f[j] - 128)
            p = np.array(X.greedy_words(P, 2))[:, None]
            ref = oracle.arith(oracle.OP_SUB, 2, C[:, j, i][:, None].copy(), p)[:, 0]
            assert np.array_equal(out[:, j, i], ref)


def test_planted_mistakes_fail_the_pins(monkeypatch):
    # a dropped diagonal (pairs p + q <= 15 only): the error bound fails
    monkeypatch.setattr(Z, "MAXD", 15)
    assert _worst_bound_ratio(Z.slab_product) > Fraction(1, 2 ** 107)
    monkeypatch.undo()
    # unbalanced digits in [0, 255]: outside the range bf16 holds exactly
    def unbalanced(x):
        a = [0] * Z.NDIG
        for p in range(Z.NDIG - 1, 0, -1):
            a[p] = x & 0xFF
            x >>= 8
        a[0] = x
        return a
    bad = unbalanced(-12345678901234567)
    assert sum(d * 256 ** (14 - p) for p, d in enumerate(bad)) == -12345678901234567
    assert not all(-128 <= d <= 127 for d in bad[1:])
