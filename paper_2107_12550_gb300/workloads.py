"""Seeded synthetic inputs shaped like the paper's benchmark problems.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle's tests.  It holds none of the method's arithmetic: no multiword
floating-point operation, no elimination, no substitution.  Matrices are built
with numpy (uniform draws, Householder QR of Gaussian matrices) and exact
integer arithmetic; the right-hand sides b = A x_true are formed exactly in
integers (or with ``math.fsum``, which returns the correctly rounded exact
sum) and then rounded greedily to binary64 words.

Conventions: a matrix of w-word values is a float64 array of shape
(w, n, lda), ``A[c, j, i]`` = word c of A(i, j) (component planes,
column-major); a vector is (w, n).  Seeds feed ``numpy.random.Generator
(PCG64(seed))``.

Workloads (the paper's own generator is Section 3, Eq. (1): A = R D R^-1 with
d_i = 10^(-26(i-1)/n) and x = [0 1 ... n-1]^T):

* ``uniform``: entries uniform in [-1, 1) as the leading word, each further
  word drawn uniformly below half of a quarter-ulp-safe bound of the word
  above, so that the stored words are already canonical;
* ``svd``: A = U diag(sigma) V^T with U, V the Q factors of Householder QR of
  Gaussian matrices, quantised to multiples of 2^-20, and sigma_k =
  2^(-round(k E/(n-1))), E = round(log2 kappa): A is formed exactly and
  rounded to words, b = A x_true is exact in 8 words, so x* = x_true;
* ``paper``: the same construction with U = V = R (so A = R D R^T, R
  orthogonal) and D = diag(2^(-round(log2(10) 26 (i-1)/n))), x = [0..n-1].
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_LB = 20                      # limb width (bits) of the exact integer pipeline
_LMASK = (1 << _LB) - 1


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def pad_lda(n: int, align: int = 32) -> int:
    """Leading dimension padded to a multiple of ``align`` doubles (256 B)."""
    return max(align, ((n + align - 1) // align) * align)


# ---------------------------------------------------------------------------
# uniform matrices
# ---------------------------------------------------------------------------

def _lower_word(g: np.random.Generator, above: np.ndarray) -> np.ndarray:
    """A word drawn uniformly in (-2^(e-54), 2^(e-54)), e = exponent of the
    word above: strictly below every rounding boundary of the word above, so
    (above, new) is canonical without any renormalisation."""
    u = g.uniform(-1.0, 1.0, size=above.shape)
    _, ex = np.frexp(above)                   # above = f 2^ex, f in [0.5, 1)
    lo = np.ldexp(u, ex - 1 - 54)
    return np.where(above == 0.0, 0.0, lo)


def uniform_matrix(n: int, words: int = 2, seed: int = 0, lda: Optional[int] = None) -> np.ndarray:
    """A(i, j) leading word ~ U[-1, 1); lower words as in ``_lower_word``."""
    lda = lda or pad_lda(n)
    g = rng(seed)
    A = np.zeros((words, n, lda))
    A[0, :, :n] = g.uniform(-1.0, 1.0, size=(n, n))
    for c in range(1, words):
        A[c, :, :n] = _lower_word(g, A[c - 1, :, :n])
    return A


def rowsum_words(A: np.ndarray, x: Optional[np.ndarray] = None, nw: int = 2) -> np.ndarray:
    """b = A x rounded greedily to nw words, via ``math.fsum`` (exact sum,
    correctly rounded).  x is a vector of small integers given as float
    (products a*x_j must be exact doubles; default x = ones)."""
    w, n = A.shape[0], A.shape[1]
    b = np.zeros((nw, n))
    if x is None:
        terms_all = A[:, :, :n].transpose(2, 0, 1).reshape(n, w * n)   # row i: all words
    else:
        prod = A[:, :, :n] * x[None, :, None]
        chk = prod / np.where(x[None, :, None] == 0, 1.0, x[None, :, None])
        assert np.array_equal(np.where(x[None, :, None] == 0, A[:, :, :n], chk), A[:, :, :n])
        terms_all = prod.transpose(2, 0, 1).reshape(n, w * n)
    for i in range(n):
        terms = terms_all[i].tolist()
        for c in range(nw):
            v = math.fsum(terms)
            b[c, i] = v
            terms.append(-v)
    return b


# ---------------------------------------------------------------------------
# exact integer pipeline (limbs of _LB bits, int64, vectorised)
# ---------------------------------------------------------------------------

def _limb_norm(L: np.ndarray) -> np.ndarray:
    """Carry-normalise limbs (axis 0, least significant first): limbs below
    the top in [0, 2^_LB), the top limb signed."""
    L = L.copy()
    for k in range(L.shape[0] - 1):
        c = L[k] >> _LB
        L[k] -= c << _LB
        L[k + 1] += c
    return L


def _rn_take(L: np.ndarray):
    """One greedy step on normalised limbs: returns (c, L') with c the
    binary64 nearest (ties to even) to the integer M = sum L_k 2^(_LB k),
    and L' the normalised limbs of M - c.  |M| < 2^1000 assumed."""
    K, N = L.shape
    neg = L[K - 1] < 0
    Lm = np.where(neg[None, :], -L, L)
    Lm = _limb_norm(Lm)
    nz = Lm != 0
    anynz = nz.any(axis=0)
    t = np.where(anynz, K - 1 - np.argmax(nz[::-1], axis=0), 0)
    cols = np.arange(N)

    def limb(idx):
        ok = idx >= 0
        return np.where(ok, Lm[np.clip(idx, 0, K - 1), cols], 0).astype(np.uint64)

    mt = limb(t)
    _, h = np.frexp(mt.astype(np.float64))      # bit length of the top limb
    h = h.astype(np.int64)
    hi = (limb(t) << np.uint64(_LB)) | limb(t - 1)           # h + 20 bits
    lo = (limb(t - 2) << np.uint64(_LB)) | limb(t - 3)       # 40 bits
    sh_hi = (33 - h).astype(np.uint64)
    sh_lo = (7 + h).astype(np.uint64)
    q = (hi << sh_hi) | (lo >> sh_lo)                         # top 53 bits
    rbit = (lo >> (sh_lo - np.uint64(1))) & np.uint64(1)
    sticky = (lo & ((np.uint64(1) << (sh_lo - np.uint64(1))) - np.uint64(1))) != 0
    below = np.zeros(N, dtype=bool)
    for k in range(K):
        below |= (Lm[k] != 0) & (k < t - 3)
    sticky |= below
    q = q + (rbit & ((sticky.astype(np.uint64)) | (q & np.uint64(1))))
    lsb = _LB * (t - 3) + 7 + h                               # weight of q's lsb
    # numbers with at most 53 bits are exact: q covers them directly
    small = (_LB * t + h) <= 53
    exact_val = np.zeros(N, dtype=np.int64)
    for k in range(min(K, 3)):
        exact_val += Lm[k] << (_LB * k)
    c_mag = np.where(small, exact_val.astype(np.float64),
                     np.ldexp(q.astype(np.float64), lsb))
    c_mag = np.where(anynz, c_mag, 0.0)
    # subtract c from the magnitude limbs
    R = Lm.copy()
    sub_q = np.where(small, exact_val.astype(np.uint64), q)
    sub_lsb = np.where(small, 0, lsb)
    j0 = sub_lsb // _LB
    r0 = (sub_lsb % _LB).astype(np.uint64)
    for part in range(3):
        chunk = (sub_q >> np.uint64(_LB * part)) & np.uint64(_LMASK)
        v = (chunk << r0).astype(np.int64)                    # < 2^40
        idx = j0 + part
        ok = anynz & (idx < K)
        R[idx[ok], cols[ok]] -= v[ok]      # one (limb, column) pair per column: no repeats
    R = _limb_norm(R)
    R = np.where(neg[None, :], -R, R)
    R = _limb_norm(R)
    c = np.where(neg, -c_mag, c_mag)
    return c, R


def _limbs_to_words(L: np.ndarray, nw: int, scale_exp: int) -> np.ndarray:
    """Greedy RN words of 2^scale_exp * M for the integers M held in limbs."""
    L = _limb_norm(L)
    out = np.zeros((nw, L.shape[1]))
    for c in range(nw):
        v, L = _rn_take(L)
        out[c] = np.ldexp(v, scale_exp)
    return out


def _exact_usv(U: np.ndarray, V: np.ndarray, e: np.ndarray, E: int, K: int) -> np.ndarray:
    """Limbs of M = sum_k U_ik V_jk 2^(E - e_k) for integer matrices U, V
    (|entries| <= 2^20) and integer exponents 0 <= e_k <= E.
    Returns int64 limbs of shape (K, n*n) in column-major element order."""
    n = U.shape[0]
    L = np.zeros((K, n * n), dtype=np.int64)
    for ev in np.unique(e):
        idx = np.nonzero(e == ev)[0]
        for s in range(0, idx.size, 1024):          # keeps every BLAS sum < 2^53
            cols = idx[s:s + 1024]
            Tf = U[:, cols] @ V[:, cols].T           # exact: integer sums < 2^52
            T = np.rint(Tf).astype(np.int64).T.reshape(-1)   # column-major (j, i)
            shift = int(E - ev)
            q, r = divmod(shift, _LB)
            t0 = T & _LMASK
            t1 = (T >> _LB) & _LMASK
            t2 = T >> (2 * _LB)
            L[q] += t0 << r
            L[q + 1] += t1 << r
            L[q + 2] += t2 << r
    return L


def _orthogonal_q20(g: np.random.Generator, n: int) -> np.ndarray:
    """Q factor of Householder QR of an n x n Gaussian matrix, quantised to
    integers (multiples of 2^-20 scaled by 2^20), as float64 integers."""
    G = g.standard_normal((n, n))
    Q, R = np.linalg.qr(G)
    Q = Q * np.sign(np.diag(R))[None, :]             # unique Haar-distributed Q
    return np.rint(Q * 2.0 ** 20)


@dataclass
class System:
    """A linear system A x = b with known exact solution x_star (or None)."""
    A: np.ndarray          # (wa, n, lda)
    b: np.ndarray          # (wb, n)
    x_star: Optional[np.ndarray]   # (n,) float64 when exactly representable
    kappa_log2: Optional[float] = None
    name: str = ""


def svd_system(n: int, log10_kappa: float, seed: int = 0, words: int = 4,
               b_words: int = 8, lda: Optional[int] = None) -> System:
    """A = U diag(sigma) V^T with sigma geometric from 1 to ~kappa (powers of
    two), formed exactly and rounded to ``words`` words; b = A * ones exactly
    (in ``b_words`` words it is exact), so x* = ones."""
    lda = lda or pad_lda(n)
    g = rng(seed)
    E = int(round(math.log2(10.0) * log10_kappa))
    U = _orthogonal_q20(g, n)
    V = _orthogonal_q20(g, n)
    e = np.rint(np.arange(n) * (E / max(n - 1, 1))).astype(np.int64)
    K = (42 + 12 + E) // _LB + 5
    L = _limb_norm(_exact_usv(U, V, e, E, K))
    S = 40 + E                                       # A = M 2^-S
    Aw = _limbs_to_words(L, words, -S)               # (words, n*n), column-major
    A = np.zeros((words, n, lda))
    A[:, :, :n] = Aw.reshape(words, n, n)
    Lb = L.reshape(K, n, n).sum(axis=1)              # sum over j: exact row sums
    b = _limbs_to_words(Lb, b_words, -S)
    return System(A, b, np.ones(n), float(E), f"svd n={n} kappa=2^{E}")


def paper_system(n: int, seed: int = 0, words: int = 4, b_words: int = 8,
                 lda: Optional[int] = None, digits: float = 26.0) -> System:
    """Section 3, Eq. (1): A = R D R^T (R orthogonal, so R^-1 = R^T),
    d_i = 10^(-26(i-1)/n) rounded to powers of two, x = [0, 1, ..., n-1]^T,
    b = A x exact in ``b_words`` words."""
    lda = lda or pad_lda(n)
    g = rng(seed)
    R = _orthogonal_q20(g, n)
    e = np.rint(np.arange(n) * (math.log2(10.0) * digits / n)).astype(np.int64)
    E = int(e.max())
    K = (42 + 12 + E + 12) // _LB + 5
    L = _limb_norm(_exact_usv(R, R, e, E, K))
    S = 40 + E
    Aw = _limbs_to_words(L, words, -S)
    A = np.zeros((words, n, lda))
    A[:, :, :n] = Aw.reshape(words, n, n)
    xs = np.arange(n, dtype=np.int64)
    Lb = (L.reshape(K, n, n) * xs[None, :, None]).sum(axis=1)
    b = _limbs_to_words(Lb, b_words, -S)
    return System(A, b, xs.astype(np.float64), float(E), f"paper n={n}")


def uniform_system(n: int, words: int = 2, seed: int = 0, b_words: int = 2,
                   lda: Optional[int] = None) -> System:
    """Uniform A; b = A * ones rounded to b_words words (x* is then the exact
    solution of the stored system, not ones, unless b_words is large)."""
    A = uniform_matrix(n, words, seed, lda)
    b = rowsum_words(A, None, b_words)
    return System(A, b, None, None, f"uniform n={n} w={words}")


# ---------------------------------------------------------------------------
# batches of uneven systems
# ---------------------------------------------------------------------------

def batch_sizes(count: int, n_lo: int, n_hi: int, seed: int = 0) -> np.ndarray:
    """n_i uniform in [n_lo, n_hi] (inclusive)."""
    return rng(seed).integers(n_lo, n_hi + 1, size=count).astype(np.int64)


def system_seed(seed: int, index: int) -> int:
    return seed * (1 << 32) + index


# ---------------------------------------------------------------------------
# mixed-precision batched refinement workload: many SVD systems of uneven
# order with log-uniform condition numbers
# ---------------------------------------------------------------------------

def mixed_batch_spec(count: int = 512, n_lo: int = 64, n_hi: int = 1024, log10_kappa_lo: float = 4.0,
                     log10_kappa_hi: float = 20.0, seed: int = 0):
    """(n_list, log10_kappa_list): n_i uniform in [n_lo, n_hi], log10 kappa_i
    uniform in [log10_kappa_lo, log10_kappa_hi]."""
    n_list = [int(v) for v in batch_sizes(count, n_lo, n_hi, seed=seed)]
    kap = rng(system_seed(seed, 1 << 31)).uniform(log10_kappa_lo, log10_kappa_hi, count)
    return n_list, [float(k) for k in kap]


def _svd_batch_worker(job):
    from multiprocessing import shared_memory
    (shm_a, shm_b, total_a, total_b, a_words, b_words, seed, items) = job
    sa = shared_memory.SharedMemory(name=shm_a)
    sb = shared_memory.SharedMemory(name=shm_b)
    try:
        Aflat = np.ndarray((total_a,), dtype=np.float64, buffer=sa.buf)
        bflat = np.ndarray((total_b,), dtype=np.float64, buffer=sb.buf)
        for (s, n, lk, moff, voff, sid) in items:
            sysm = svd_system(n, lk, seed=system_seed(seed, sid), words=a_words, b_words=b_words, lda=n)
            base = a_words * moff
            Aflat[base: base + a_words * n * n] = sysm.A.reshape(-1)
            vb = b_words * voff
            bflat[vb: vb + b_words * n] = sysm.b.reshape(-1)
        return len(items)
    finally:
        del Aflat, bflat
        sa.close()
        sb.close()


def svd_batch(n_list, log10_kappa, seed: int = 0, a_words: int = 4, b_words: int = 8,
              processes: Optional[int] = None, system_ids=None):
    """Packed batch of ``svd_system`` s (system s uses seed system_seed(seed, s),
    lda = n): returns (A, b) flat float64 arrays in the batch layout (system s:
    A at a_words * sum_{s'<s} n^2, b at b_words * sum_{s'<s} n), with
    x* = ones for every system.  Systems are built in a pool of worker
    processes (spawn start method) writing into shared memory.
    system_ids: for a subset of a larger batch, the original index of each
    listed system (its seed is system_seed(seed, id)); default 0..count-1."""
    ids = list(range(len(n_list))) if system_ids is None else [int(v) for v in system_ids]
    import multiprocessing as mp
    from multiprocessing import shared_memory
    n = np.asarray(n_list, dtype=np.int64)
    moff = np.concatenate([[0], np.cumsum(n * n)])
    voff = np.concatenate([[0], np.cumsum(n)])
    total_a, total_b = a_words * int(moff[-1]), b_words * int(voff[-1])
    sa = shared_memory.SharedMemory(create=True, size=max(8, 8 * total_a))
    sb = shared_memory.SharedMemory(create=True, size=max(8, 8 * total_b))
    try:
        np.ndarray((total_a,), dtype=np.float64, buffer=sa.buf)[:] = 0.0
        np.ndarray((total_b,), dtype=np.float64, buffer=sb.buf)[:] = 0.0
        procs = processes or os.cpu_count() or 1
        order = sorted(range(len(n_list)), key=lambda s: -int(n_list[s]))
        buckets = [[] for _ in range(procs)]
        load = [0.0] * procs
        for s in order:                              # longest-processing-time first
            k = int(np.argmin(load))
            buckets[k].append((s, int(n_list[s]), float(log10_kappa[s]), int(moff[s]), int(voff[s]), ids[s]))
            load[k] += float(n_list[s]) ** 2.5
        jobs = [(sa.name, sb.name, total_a, total_b, a_words, b_words, seed, it) for it in buckets if it]
        if procs == 1:
            for j in jobs:
                _svd_batch_worker(j)
        else:
            # one BLAS thread per worker (the workers import numpy afresh and
            # read these); a worker that dies raises BrokenProcessPool here
            # instead of leaving the parent waiting
            from concurrent.futures import ProcessPoolExecutor
            keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")
            saved = {k: os.environ.get(k) for k in keys}
            try:
                for k in keys:
                    os.environ[k] = "1"
                with ProcessPoolExecutor(max_workers=len(jobs), mp_context=mp.get_context("spawn")) as ex:
                    list(ex.map(_svd_batch_worker, jobs))
            finally:
                for k, v in saved.items():
                    if v is None:
                        os.environ.pop(k, None)
                    else:
                        os.environ[k] = v
        A = np.array(np.ndarray((total_a,), dtype=np.float64, buffer=sa.buf))
        b = np.array(np.ndarray((total_b,), dtype=np.float64, buffer=sb.buf))
    finally:
        sa.close()
        sa.unlink()
        sb.close()
        sb.unlink()
    return A, b

