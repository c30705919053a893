"""mpmath interoperability (host conversions): the greedy round-to-nearest
word expansion against the oracle's, exact round trips, special values; on
the GPU, refinement of an mpmath system to 2^-200."""
import random
from fractions import Fraction

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

from oracle import exact as X  # noqa: E402
from paper_2107_12550_gb300 import mp as MP  # noqa: E402


def _rand_mpf(rng: random.Random, bits: int, emin: int = -300, emax: int = 300):
    man = rng.getrandbits(bits) | (1 << (bits - 1))
    if rng.random() < 0.5:
        man = -man
    return mpmath.mpf((man, rng.randint(emin, emax) - bits))


@pytest.mark.parametrize("w", [2, 3, 4, 8])
def test_to_words_is_the_oracle_greedy_expansion(w):
    rng = random.Random(100 + w)
    with mpmath.workprec(1200):
        for _ in range(300):
            x = _rand_mpf(rng, rng.randint(1, 1000))
            M, E = x.man * (-1 if x < 0 else 1), x.exp
            fx = Fraction(M) * (Fraction(2) ** E)
            assert MP.to_words(x, w) == X.greedy_words(fx, w)


def test_round_trip_exact_at_424_bits():
    """8 greedy words hold any value of at most 8 x 53 significant bits."""
    rng = random.Random(7)
    with mpmath.workprec(3000):
        for _ in range(200):
            x = _rand_mpf(rng, 424)
            assert MP.from_words(MP.to_words(x, 8)) == x


def test_special_values():
    assert MP.to_words(0, 3) == [0.0, 0.0, 0.0]
    assert MP.to_words(-1, 2) == [-1.0, 0.0]
    with mpmath.workprec(300):
        # ties to even: 1 + 2^-53 -> 1, remainder 2^-53; 1 + 3 2^-53 -> 1 + 2^-51
        assert MP.to_words(mpmath.mpf(1) + mpmath.ldexp(1, -53), 2) == [1.0, 2.0 ** -53]
        assert MP.to_words(mpmath.mpf(1) + 3 * mpmath.ldexp(1, -53), 2) == [1.0 + 2.0 ** -51, -(2.0 ** -53)]
        # the largest double and the subnormal range
        big = mpmath.ldexp(2 ** 53 - 1, 1023 - 52)
        assert MP.to_words(big, 2) == [1.7976931348623157e308, 0.0]
        tiny = mpmath.ldexp(3, -1076)                  # 0.75 x 2^-1074: rounds to 2^-1074
        assert MP.to_words(tiny, 2) == [5e-324, 0.0]   # the remainder is below the subnormal grid
        with pytest.raises(OverflowError):
            MP.to_words(mpmath.ldexp(1, 1024), 2)
    with pytest.raises(ValueError):
        MP.to_words(mpmath.inf, 2)


def test_planes_layout():
    with mpmath.workprec(200):
        A = mpmath.matrix([[1, 2], [3, mpmath.mpf(1) / 3]])
        P = MP.matrix_to_planes(A, 3, lda=4)
    assert P.shape == (3, 2, 4)
    assert P[0, 0, 1] == 3.0 and P[0, 1, 0] == 2.0          # word 0 of A(1, 0) and A(0, 1)
    assert P[0, 1, 1] == 1.0 / 3 and P[1, 1, 1] != 0.0
    with mpmath.workprec(200):
        v = MP.planes_to_vector(np.array([[1.0, 2.0], [2.0 ** -60, 0.0]]))
        assert v[0] == 1 + mpmath.ldexp(1, -60) and v[1] == 2
    v53 = MP.planes_to_vector(np.array([[1.0], [2.0 ** -60]]))   # rounded to the 53-bit default
    assert v53[0] == 1


@pytest.mark.gpu
def test_refine_mp_to_2_pow_minus_200():
    """An mpmath system (integer matrix, b = A * ones exactly): the GPU
    refinement with a TD inner LU returns x = ones within 2^-200."""
    pytest.importorskip("torch")
    from paper_2107_12550_gb300 import build as B
    B.build()
    n = 40
    rng = np.random.default_rng(3)
    M = rng.integers(-9, 10, (n, n))
    M += np.diag(np.full(n, 60))
    A = mpmath.matrix(M.tolist())
    b = mpmath.matrix([sum(int(v) for v in M[i]) for i in range(n)])
    with mpmath.workprec(600):
        x, res = MP.refine_mp(A, b, inner_prec=3, target_bits=200)
        assert res.status == 0
        for i in range(n):
            assert abs(x[i] - 1) <= mpmath.ldexp(1, -200)
