"""mpmath interoperability: mpmath matrices and vectors in and out of the
multiword (w-word binary64) planes the library computes on.

The paper drives its DD/TD/QD routines from mpmath matrices (Section 2 and its
listing: the matrix is converted to the short format, factored, the residual
formed in mpmath, and the correction converted back).  Here the conversions
are exact host-side integer arithmetic:

* ``to_words(x, w)`` is the greedy round-to-nearest expansion
  c_i = RN(x - c_0 - ... - c_{i-1}), i = 0..w-1 (ties to even);
* ``from_words(c)`` is the exact sum of the words, returned as an mpf rounded
  to the current mpmath precision (exact when that precision spans it);
* ``ludecomp_mp``, ``solve_mp`` and ``refine_mp`` wrap the GPU calls of
  ``api`` for mpmath inputs and outputs.

This is interface code around the device path: every arithmetic step of the
factorisation, substitution and refinement still runs in the CUDA library.
"""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import numpy as np

_EMIN = -1074          # exponent of the smallest subnormal
_EMAX = 1023           # exponent of the largest binary64 binade


def _man_exp(x) -> Tuple[int, int]:
    """x as an exact (signed integer M, exponent E) with x = M 2^E."""
    import mpmath
    if isinstance(x, float):
        if not math.isfinite(x):
            raise ValueError("non-finite value")
        m, e = math.frexp(x)
        return int(m * (1 << 53)), e - 53
    if isinstance(x, int):
        return x, 0
    v = x if isinstance(x, mpmath.mpf) else mpmath.mpf(x)
    if not mpmath.isfinite(v):
        raise ValueError("non-finite value")
    if v == 0:
        return 0, 0
    sign, man, exp, _ = v._mpf_
    return (-int(man) if sign else int(man)), int(exp)


def _rn_double(M: int, E: int) -> Tuple[float, int]:
    """RN(M 2^E) as a double d, and the exact remainder's integer
    mantissa R with M 2^E - d = R 2^E (on the same exponent E)."""
    if M == 0:
        return 0.0, 0
    a = -M if M < 0 else M
    top = E + a.bit_length() - 1                 # value in [2^top, 2^(top+1))
    q = max(top - 52, _EMIN)                     # exponent of the last kept bit
    if E >= q:
        if top > _EMAX:
            raise OverflowError("value beyond the binary64 range")
        d = math.ldexp(float(a), E)              # a < 2^53 here: exact
        return (-d if M < 0 else d), 0
    sh = q - E
    r = a >> sh
    rem = a - (r << sh)
    half = 1 << (sh - 1)
    if rem > half or (rem == half and (r & 1)):
        r += 1
    if q + r.bit_length() - 1 > _EMAX:
        raise OverflowError("value beyond the binary64 range")
    d = math.ldexp(float(r), q)                  # r <= 2^53: exact
    R = a - (r << sh)
    return (-d, -R) if M < 0 else (d, R)


def to_words(x, w: int) -> List[float]:
    """The w-word greedy round-to-nearest expansion of x (an mpf, int,
    float, or anything mpmath.mpf accepts at the current precision)."""
    M, E = _man_exp(x)
    out = []
    for _ in range(w):
        d, M = _rn_double(M, E)
        out.append(d)
    return out


def _words_man_exp(words: Sequence[float]) -> Tuple[int, int]:
    parts = [_man_exp(float(c)) for c in words if c != 0.0]
    if not parts:
        return 0, 0
    e0 = min(e for _, e in parts)
    return sum(m << (e - e0) for m, e in parts), e0


def from_words(words: Sequence[float]):
    """The exact sum of the words as an mpf at the current mpmath precision."""
    import mpmath
    M, E = _words_man_exp(words)
    return mpmath.mpf((M, E)) if M else mpmath.mpf(0)


def matrix_to_planes(A, w: int, lda: int = 0) -> np.ndarray:
    """An n x n mpmath matrix (or nested sequences) as the library's planes:
    shape (w, n, lda), word c of A(i, j) at [c, j, i]."""
    n = A.rows if hasattr(A, "rows") else len(A)
    lda = lda or n
    P = np.zeros((w, n, lda))
    for i in range(n):
        for j in range(n):
            v = A[i, j] if hasattr(A, "rows") else A[i][j]
            P[:, j, i] = to_words(v, w)
    return P


def vector_to_planes(b, w: int) -> np.ndarray:
    """An mpmath column vector (or a sequence) as planes of shape (w, n)."""
    n = b.rows if hasattr(b, "rows") else len(b)
    P = np.zeros((w, n))
    for i in range(n):
        P[:, i] = to_words(b[i], w)
    return P


def planes_to_vector(x: np.ndarray):
    """Planes (w, n) back to an mpmath column vector (exact sums, rounded to
    the current precision)."""
    import mpmath
    w, n = x.shape
    return mpmath.matrix([from_words(x[:, i]) for i in range(n)])


def ludecomp_mp(A, prec: int = 3):
    """LU with partial pivoting of an mpmath matrix at w = prec words on the
    GPU.  Returns (LU planes as a cuda tensor (w, n, n), pivots, info)."""
    import torch
    from . import api
    planes = matrix_to_planes(A, prec)
    return api.ludecomp(torch.from_numpy(planes).cuda(), prec)


def solve_mp(LU, piv, b, prec: int = 3):
    """Forward/back substitution on the GPU for an mpmath right-hand side;
    returns an mpmath vector."""
    import torch
    from . import api
    x = api.solve(LU, piv, torch.from_numpy(vector_to_planes(b, prec)).cuda(), prec)
    return planes_to_vector(x.cpu().numpy())


def refine_mp(A, b, inner_prec: int = 3, target_bits: int = 200, a_words: int = 4, update: str = "plain",
              **kw):
    """Mixed-precision iterative refinement of an mpmath system on the GPU:
    A rounded to a_words words, b to 8 words, the inner LU at inner_prec
    words, refined until the target relative error bound is met.  Returns
    (x as an mpmath vector, the library's RefineResult)."""
    import torch
    from . import api
    Ap = torch.from_numpy(matrix_to_planes(A, a_words)).cuda()
    bp = torch.from_numpy(vector_to_planes(b, 8)).cuda()
    res = api.refine(Ap, bp, inner_prec, target_bits, update=update, **kw)
    return planes_to_vector(res.x.cpu().numpy()), res
