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
Planted mistakes in the model (a dropped diagonal, unbalanced digits, a
scale one bit short, a dropped low word, a recombination shifted by one
digit, an exact form without its second word) are shown to fail these
pins."""
import math
import os
import types
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


def _model_variant(old: str, new: str):
    """A copy of the model with one planted mistake (the text `old`, which
    must occur once, replaced by `new`), loaded as a module of the oracle
    package so that its relative imports resolve."""
    path = os.path.join(os.path.dirname(Z.__file__), "ozaki.py")
    src = open(path).read()
    assert src.count(old) == 1, old
    mod = types.ModuleType("oracle.ozaki_variant")
    mod.__package__ = "oracle"
    exec(compile(src.replace(old, new), path + " (variant)", "exec"), mod.__dict__)
    return mod


def _scaled_entries_in_range(model):
    """Step 1's invariant: every scaled entry lies in (-1/2, 1/2), i.e. its
    integer on the 2^-120 grid stays below 2^119 in magnitude (the digit
    ranges and the FP32 exactness bound rest on it)."""
    g = np.random.default_rng(5)
    L = _dd_random(g, 16, 64, scale_rows=True)
    for i in range(16):
        e = model.scale_exponent(L[0, :, i])
        for t in range(64):
            X = model.floor_scaled(L[0, t, i], model.GRID - e) + model.floor_scaled(L[1, t, i], model.GRID - e)
            if abs(X) >= 2 ** 119:
                return False
    return True


def _exact_form_two_words(model):
    """C with both words on the product's grid, a large hi and a small lo:
    C - L U needs both result words, and the exact form must give the
    greedy DD rounding of the exact value."""
    g = np.random.default_rng(6)
    m, N, K = 4, 3, 64
    L = np.zeros((2, K, m)); L[0] = g.integers(-100, 101, (K, m))
    U = np.zeros((2, N, K)); U[0] = g.integers(-100, 101, (N, K))
    C = np.zeros((2, N, m))
    C[0] = 2.0 ** 40 * g.choice([-1.0, 1.0], (N, m))
    C[1] = 2.0 ** -20 * g.integers(1, 100, (N, m))
    out, nexact = model.update(C, L, U, m, N, K)
    if nexact != m * N:
        return False
    for i in range(m):
        for j in range(N):
            v = X.words_to_frac(C[:, j, i]) - _exact_prod(L, U, i, j, K)
            if list(out[:, j, i]) != X.greedy_words(v, 2):
                return False
    return True


def _small_integers_exact(model):
    g = np.random.default_rng(2)
    m, N, K = 9, 7, 64
    L = np.zeros((2, K, m)); L[0] = g.integers(-100, 101, (K, m))
    U = np.zeros((2, N, K)); U[0] = g.integers(-100, 101, (N, K))
    R, e, f = model.slab_product(L, U, m, N, K)
    return all(R[i][j] * Fraction(2) ** (e[i] + f[j] - 128) == _exact_prod(L, U, i, j, K)
               for i in range(m) for j in range(N))


MODEL_MUTATIONS = [
    ("scale exponent one bit short", "    return _ilogb(mx) + 2 if mx != 0.0 else 0\n",
     "    return _ilogb(mx) + 1 if mx != 0.0 else 0\n", _scaled_entries_in_range),
    ("recombination shifted by one digit",
     "    R = [[sum(int(D[d][i, j]) << (8 * (MAXD - d)) for d in range(2, MAXD + 1)) for j in range(N)]\n",
     "    R = [[sum(int(D[d][i, j]) << (8 * (MAXD - d + 1)) for d in range(2, MAXD + 1)) for j in range(N)]\n",
     _small_integers_exact),
    ("row operand's low word dropped",
     "            X = floor_scaled(L[0, t, i], GRID - e[i]) + floor_scaled(L[1, t, i], GRID - e[i])\n",
     "            X = floor_scaled(L[0, t, i], GRID - e[i])\n",
     lambda model: _worst_bound_ratio(model.slab_product) <= Fraction(1, 2 ** 107)),
    ("exact form without its second word", "                    lo = _rn(V - Fraction(hi))\n",
     "                    lo = 0.0\n", _exact_form_two_words),
]


@pytest.mark.parametrize("name,old,new,pin", MODEL_MUTATIONS, ids=[m[0] for m in MODEL_MUTATIONS])
def test_planted_model_mistake_is_caught(name, old, new, pin):
    assert pin(Z), "the pin must pass on the unmodified model"
    assert not pin(_model_variant(old, new)), name
