"""Parity rules shared by the GPU tests.

Full-size plain factorisations: the first columns against the oracle's
first elimination steps (first_columns_bitwise).

Results of the split (tensor-core) LU, which is not bitwise equal to the
oracle (only the plain path is), follow these parity rules for the split
path:

* Pivots: identical to the reference sequence (the oracle's, or the plain
  GPU path's, which the parity tests pin bitwise to the oracle) up to the
  first divergence k.  That one is accepted only as a near-tie: in the
  oracle's values after k elimination steps,
      | |a_(p_gpu, k)| - |a_(p_ref, k)| |  <=  2^-(53 w - log2 n - 10) |a_(p_ref, k)|.
  After it only the error criteria apply.
* Normwise backward error eta from an exact residual.
* Forward error within 10x the oracle's own at the same precision.

Helpers only (no tests here); the oracle is the reference throughout."""
import math
from fractions import Fraction

import numpy as np

import oracle
from oracle import exact as X


def first_divergence(piv_gpu, piv_ref):
    d = np.nonzero(np.asarray(piv_gpu) != np.asarray(piv_ref))[0]
    return int(d[0]) if d.size else None


def check_pivots_near_tie(A, w, piv_gpu, piv_ref):
    """Pivots equal to piv_ref, or equal up to a first divergence that is a
    near-tie in the oracle's values; returns the divergence step or None."""
    n = A.shape[1]
    k = first_divergence(piv_gpu, piv_ref)
    if k is None:
        return None
    LUk, pivk, _ = oracle.lu_steps(w, A, k)
    assert np.array_equal(pivk[:k], np.asarray(piv_ref)[:k])
    a_g = abs(X.words_to_frac(LUk[:w, k, int(piv_gpu[k])]))
    a_r = abs(X.words_to_frac(LUk[:w, k, int(piv_ref[k])]))
    lim = Fraction(2) ** -(53 * w - math.ceil(math.log2(max(n, 2))) - 10) * a_r
    assert abs(a_g - a_r) <= lim, f"pivot divergence at step {k} is not a near-tie"
    return k


def eta(A, b, x):
    """Normwise backward error ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)
    with the residual computed exactly (oracle) and rounded to 8 words."""
    n = x.shape[1]
    r = oracle.residual(A, b, x, 8)
    Ainf = np.max(np.sum(np.abs(A[0, :, :n]), axis=0))
    return np.max(np.abs(r[0])) / (Ainf * np.max(np.abs(x[0])) + np.max(np.abs(b[0])))


def exact_solution(A, b):
    """x* of the stored system to well below 2^-300 relative: the oracle's
    refinement with a DD inner solve and an 8-word iterate."""
    st, x, corr, nres, info = oracle.refine(A, b, 2, target_bits=320, max_iter=60)
    assert st == 0 and info == 0
    return X.vec_to_frac(x)


def forward_error(x, xstar):
    return X.forward_error(X.vec_to_frac(x), xstar)


def first_columns_bitwise(A, w, LUg, pivg, ks=8):
    """The first ks columns of a full-size GPU factorisation against the
    oracle's first ks elimination steps: pivots 0..ks-1 equal, and columns
    0..ks-1 equal bitwise once the GPU's later row swaps are applied to the
    oracle's (those columns are final after step ks-1 up to the swaps)."""
    n = A.shape[1]
    LUo, pivo, _ = oracle.lu_steps(w, A, ks)
    assert np.array_equal(pivg[:ks], pivo[:ks])
    cols = LUo[:w, :ks, :n].copy()
    for k in range(ks, n):
        p = int(pivg[k])
        if p != k:
            cols[:, :, [k, p]] = cols[:, :, [p, k]]
    assert np.array_equal(LUg[:w, :ks, :n], cols)
