"""CPU oracle for multiword (DD/TD/QD) LU, substitution, exact residual and
mixed-precision iterative refinement.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the library under
``paper_2107_12550_gb300`` never does, and this package never imports it.

Two independent parts:

* ``mwo.c`` (wrapped here with ctypes): plain C, compiled with
  ``-O2 -ffp-contract=off -fno-fast-math``; DD/TD/QD arithmetic, unblocked LU
  with partial pivoting, substitution, the exact residual and the refinement
  loop of the paper (Section 2, Listing 1; stopping test Eq. (2)).
* ``exact.py``: pure-Python ``fractions.Fraction`` arithmetic (exact Gaussian
  elimination, exact residuals, greedy rounding) used to pin ``mwo.c``.

Array conventions (numpy, float64, C order): a matrix of w-word values has
shape ``(w, n, lda)`` with ``A[c, j, i]`` = word c of A(i, j) (component
planes, column-major); a vector has shape ``(w, n)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mwo.c")
_LIB = os.path.join(_HERE, "libmwo.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile ``mwo.c`` into ``libmwo.so`` next to it (no-op when current)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.run(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _bind(path: str) -> ctypes.CDLL:
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    I = ctypes.c_int
    D = ctypes.c_double
    L.mwo_eft.argtypes = [I, I64, P, P, P, P]
    L.mwo_arith.argtypes = [I, I, I64, P, P, P]
    L.mwo_lu.argtypes = [I, I64, P, I64, P, P]
    L.mwo_lu_steps.argtypes = [I, I64, P, I64, P, P, I64]
    L.mwo_solve.argtypes = [I, I64, P, I64, P, P, P]
    L.mwo_residual.argtypes = [I64, P, I64, I, P, I, P, I, P, I]
    L.mwo_exact_sum.argtypes = [I64, P, I, P]
    L.mwo_exact_dot.argtypes = [I64, P, P, I, P]
    L.mwo_refine.argtypes = [I64, P, I64, I, P, I, I, I, I, D, D, I, P, I, P]
    L.mwo_set_threads.argtypes = [I]
    for f in ("mwo_eft", "mwo_arith", "mwo_lu", "mwo_lu_steps", "mwo_solve", "mwo_residual",
              "mwo_exact_sum", "mwo_exact_dot", "mwo_refine", "mwo_set_threads"):
        getattr(L, f).restype = I
    return L


def lib() -> ctypes.CDLL:
    """The oracle library in use (built on first use)."""
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _bind(_LIB)
    return _lib


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile a (possibly mutated) copy of the oracle source to out_path;
    used by the tests that plant mistakes to show the pins catch them."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", *CFLAGS, "-o", out_path, src, "-lm"], check=True)
    return out_path


class use:
    """Context manager: route the module-level functions to another build
    of the oracle (a planted-mistake variant) for the duration."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        lib()
        self._saved = _lib
        _lib = _bind(self.path)
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _p(a: np.ndarray) -> int:
    assert a.flags.c_contiguous
    return a.ctypes.data


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(t: int = 0) -> int:
    """Set the OpenMP thread count (0 keeps it); returns the count in use."""
    return lib().mwo_set_threads(int(t))


EFT_TWOSUM, EFT_FASTTWOSUM, EFT_TWOPROD = 0, 1, 2


def eft(op: int, a, b):
    a = _f64(a).ravel()
    b = _f64(b).ravel()
    s = np.empty_like(a)
    e = np.empty_like(a)
    rc = lib().mwo_eft(op, a.size, _p(a), _p(b), _p(s), _p(e))
    assert rc == 0
    return s, e


OP_ADD, OP_SUB, OP_MUL, OP_DIV, OP_CMPABS, OP_MULD, OP_RENORM = range(7)


def arith(op: int, w: int, x, y):
    """Element-wise multiword op on arrays of shape (w, cnt); for OP_MULD, y
    has shape (cnt,).  OP_CMPABS returns an int array (cnt,)."""
    x = _f64(x)
    y = _f64(y)
    cnt = x.shape[1]
    z = np.zeros((w, cnt))
    rc = lib().mwo_arith(op, w, cnt, _p(x), _p(y), _p(z))
    assert rc == 0, rc
    if op == OP_CMPABS:
        return z[0].astype(np.int64)
    return z


def lu(w: int, A):
    """Unblocked LU with partial pivoting on the first w words of A.
    Returns (LU (w, n, lda), piv int64 (n,), info)."""
    A = _f64(A)
    n, lda = A.shape[1], A.shape[2]
    LU = np.zeros((w, n, lda))
    k = min(w, A.shape[0])
    LU[:k] = A[:k]
    piv = np.zeros(max(n, 1), dtype=np.int64)
    info = np.zeros(1, dtype=np.int64)
    rc = lib().mwo_lu(w, n, _p(LU), lda, _p(piv), _p(info))
    assert rc == 0, rc
    return LU, piv[:n], int(info[0])


def lu_steps(w: int, A, ksteps: int):
    """The first ksteps elimination steps of ``lu`` (for timing samples)."""
    A = _f64(A)
    n, lda = A.shape[1], A.shape[2]
    LU = np.zeros((w, n, lda))
    k = min(w, A.shape[0])
    LU[:k] = A[:k]
    piv = np.zeros(max(n, 1), dtype=np.int64)
    info = np.zeros(1, dtype=np.int64)
    rc = lib().mwo_lu_steps(w, n, _p(LU), lda, _p(piv), _p(info), int(ksteps))
    assert rc == 0, rc
    return LU, piv[:n], int(info[0])


def solve(w: int, LU, piv, b):
    LU = _f64(LU)
    n, lda = LU.shape[1], LU.shape[2]
    piv = np.ascontiguousarray(piv, dtype=np.int64)
    bb = np.zeros((w, n))
    k = min(w, b.shape[0])
    bb[:k] = b[:k]
    x = np.zeros((w, n))
    rc = lib().mwo_solve(w, n, _p(LU), lda, _p(piv), _p(bb), _p(x))
    assert rc == 0, rc
    return x


def residual(A, b, x, wr: int = 8):
    """r = b - A x exactly, rounded greedily to wr words."""
    A = _f64(A)
    b = _f64(b)
    x = _f64(x)
    n, lda = A.shape[1], A.shape[2]
    r = np.zeros((wr, n))
    rc = lib().mwo_residual(n, _p(A), lda, A.shape[0], _p(b), b.shape[0],
                            _p(x), x.shape[0], _p(r), wr)
    assert rc == 0, rc
    return r


def exact_sum(terms, nw: int):
    t = _f64(terms).ravel()
    out = np.zeros(nw)
    assert lib().mwo_exact_sum(t.size, _p(t), nw, _p(out)) == 0
    return out


def exact_dot(x, y, nw: int):
    x = _f64(x).ravel()
    y = _f64(y).ravel()
    out = np.zeros(nw)
    assert lib().mwo_exact_dot(x.size, _p(x), _p(y), nw, _p(out)) == 0
    return out


STOP_EQ2, STOP_BITS = 0, 1


def refine(A, b, w_in: int, *, max_iter: int = 30, stop_mode: int = STOP_BITS,
           rtol: float = 1e-100, atol: float = 0.0, target_bits: int = 200, wx: int = 8):
    """Mixed precision iterative refinement (Section 2, Listing 1).
    Returns (status, x (wx, n), corrections, residuals, info)."""
    A = _f64(A)
    b = _f64(b)
    n, lda = A.shape[1], A.shape[2]
    x = np.zeros((wx, n))
    stats = np.zeros(3, dtype=np.int64)
    st = lib().mwo_refine(n, _p(A), lda, A.shape[0], _p(b), b.shape[0], w_in, max_iter,
                          stop_mode, rtol, atol, target_bits, _p(x), wx, _p(stats))
    assert st >= 0, st
    return st, x, int(stats[0]), int(stats[1]), int(stats[2])
