"""Oracle for the block matrix product and its Strassen form (Section 2:
BNCmatmul, the paper's multiword matmul, and its Strassen variant).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Built from the
oracle's own element-wise multiword operations (``oracle.arith``, the C
arithmetic pinned elsewhere), in plain loops:

* ``product(w, A, B, C0=None)``: c_ij = c0_ij + a_i0 b_0j + ... + a_i,K-1
  b_K-1,j accumulated in ascending t, each term a rounded multiword multiply
  followed by a rounded addition (from zero when C0 is None);
* ``strassen(w, A, B, levels)``: Strassen's seven-product recursion (Strassen
  1969) with the additions in this order, then ``product`` on the blocks:
    M1 = (A11 + A22)(B11 + B22)    M2 = (A21 + A22) B11
    M3 = A11 (B12 - B22)           M4 = A22 (B21 - B11)
    M5 = (A11 + A12) B22           M6 = (A21 - A11)(B11 + B12)
    M7 = (A12 - A22)(B21 + B22)
    C11 = ((M1 + M4) - M5) + M7    C12 = M3 + M5
    C21 = M2 + M4                  C22 = ((M1 - M2) + M3) + M6
  The paper does not fix the variant or the order of the additions; this is
  the reading the GPU path follows.

Matrices are numpy arrays (w, cols, rows): word c of X(i, j) at X[c, j, i].
"""
from __future__ import annotations

import numpy as np

from . import OP_ADD, OP_MUL, OP_SUB, arith


def _ew(op: int, w: int, X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    shape = X.shape
    return arith(op, w, np.ascontiguousarray(X).reshape(w, -1), np.ascontiguousarray(Y).reshape(w, -1)).reshape(shape)


def product(w: int, A: np.ndarray, B: np.ndarray, C0: np.ndarray | None = None) -> np.ndarray:
    """A: (w, K, m) (m x K), B: (w, N, K) (K x N) -> C (w, N, m)."""
    K, m = A.shape[1], A.shape[2]
    N = B.shape[1]
    C = np.zeros((w, N, m)) if C0 is None else np.array(C0[:, :N, :m], dtype=np.float64)
    for t in range(K):
        a = np.broadcast_to(A[:, t, :][:, None, :], (w, N, m))      # a_it for every column j
        b = np.broadcast_to(B[:, :, t][:, :, None], (w, N, m))      # b_tj for every row i
        C = _ew(OP_ADD, w, C, _ew(OP_MUL, w, a, b))
    return C


def strassen(w: int, A: np.ndarray, B: np.ndarray, levels: int) -> np.ndarray:
    """C = A B for n x n operands (w, n, n); n divisible by 2^levels."""
    if levels == 0:
        return product(w, A, B)
    n = A.shape[1]
    h = n // 2

    def q(X, r, c):          # quadrant at block row r, block column c
        return X[:, c * h:(c + 1) * h, r * h:(r + 1) * h]

    def add(X, Y):
        return _ew(OP_ADD, w, X, Y)

    def sub(X, Y):
        return _ew(OP_SUB, w, X, Y)

    def rec(X, Y):
        return strassen(w, np.ascontiguousarray(X), np.ascontiguousarray(Y), levels - 1)

    A11, A12, A21, A22 = q(A, 0, 0), q(A, 0, 1), q(A, 1, 0), q(A, 1, 1)
    B11, B12, B21, B22 = q(B, 0, 0), q(B, 0, 1), q(B, 1, 0), q(B, 1, 1)
    M1 = rec(add(A11, A22), add(B11, B22))
    M2 = rec(add(A21, A22), B11)
    M3 = rec(A11, sub(B12, B22))
    M4 = rec(A22, sub(B21, B11))
    M5 = rec(add(A11, A12), B22)
    M6 = rec(sub(A21, A11), add(B11, B12))
    M7 = rec(sub(A12, A22), add(B21, B22))
    C = np.zeros((w, n, n))
    C[:, 0:h, 0:h] = add(sub(add(M1, M4), M5), M7)      # C11
    C[:, h:n, 0:h] = add(M3, M5)                        # C12 (block row 0, block column 1)
    C[:, 0:h, h:n] = add(M2, M4)                        # C21
    C[:, h:n, h:n] = add(add(sub(M1, M2), M3), M6)      # C22
    return C
