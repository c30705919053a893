"""Ozaki scheme II (products over small moduli, Chinese remaindering) as an
exact CPU model of the split trailing update's alternative form, with the
counts that decide between the two schemes on the bf16 tensor path.

The trailing update's block product (Section 2, BNCmatmul) is reshaped by
the split path into products of scaled integers: row i of L21 and column j
of U12 are scaled by powers of two so that each entry becomes a signed
integer X with |X| < 2^(t-1) on a grid of t bits.  Scheme I writes X as 15
base-256 digits and sums 120 digit-pair products.  Scheme II instead takes X
modulo pairwise-coprime m_1 .. m_r, multiplies the residue matrices (exact in
FP32 while every partial sum stays below 2^24), reduces each product modulo
its m_l, and recovers the exact integer sum by Garner's mixed-radix form of
the Chinese remainder theorem.

Everything here is plain Python integers and numpy; the float32 products go
through numpy's matmul (a library sgemm, any summation order), which is the
point of the exactness check.  Nothing here is built on the device: the
counts below are why (the scheme I kernel is bound by its per-entry
recombination, and scheme II moves work from the tensor pipe into exactly
that recombination)."""
import math
import random

import numpy as np

K = 64                      # panel width: the inner dimension of one update
T_BITS = 120                # scheme I's grid: |X| < 2^119 (15 digits x 8 bits)
SCHEME_I_PAIRS = 120        # digit pairs (p, q) with p + q <= 16
SCHEME_I_DIAGONALS = 15     # exact FP32 sums recombined per output entry


def product_bits(t_bits, k):
    """Bits of modulus needed for the signed sum of k products of two
    integers below 2^(t_bits - 1) in magnitude: |S| < k 2^(2 t_bits - 2), and
    the symmetric residue range needs M > 2 |S|."""
    return 2 * (t_bits - 1) + math.ceil(math.log2(k)) + 1


def bf16_exact(v):
    """An integer is exact in bf16 when its magnitude has at most 8
    significant bits (one implicit, seven stored)."""
    v = abs(v)
    if v == 0:
        return True
    return v >> max(0, v.bit_length() - 8) << max(0, v.bit_length() - 8) == v


def moduli(limit, bits):
    """Largest-first greedy choice of pairwise-coprime moduli <= limit until
    their product reaches 2^bits."""
    out, prod = [], 1
    for m in range(limit, 1, -1):
        if all(math.gcd(m, q) == 1 for q in out):
            out.append(m)
            prod *= m
            if prod >= 1 << bits:
                return out
    raise ValueError("not enough coprime moduli below the limit")


def sym_res(x, m):
    """Residue of x modulo m in [-floor(m/2), ceil(m/2) - 1]."""
    r = x % m
    return r - m if r >= (m + 1) // 2 else r


def garner(res, ms):
    """Mixed-radix digits v with X = v0 + v1 m0 + v2 m0 m1 + ..., each
    v_i in [0, m_i): digit i costs i modular multiply-adds.  Returns the
    signed X in [-M/2, M/2) and the number of modular multiply-adds."""
    v, ops = [], 0
    for i, (r, m) in enumerate(zip(res, ms)):
        u = r % m
        for j in range(i):
            u = ((u - v[j]) * pow(ms[j], -1, m)) % m
            ops += 1
        v.append(u)
    X = 0
    for i in range(len(ms) - 1, -1, -1):
        X = X * ms[i] + v[i]
    M = math.prod(ms)
    return (X - M if X >= M // 2 else X), ops


def scheme2_product(X, Y, ms):
    """Exact integer product X Y (X: rows x K, Y: K x cols, Python ints) by
    residues, one float32 matmul per modulus, and Garner per entry."""
    rows, cols = len(X), len(Y[0])
    S = []
    for m in ms:
        A = np.array([[sym_res(x, m) for x in row] for row in X], dtype=np.float32)
        B = np.array([[sym_res(y, m) for y in row] for row in Y], dtype=np.float32)
        P = A @ B
        S.append(P)
    out, ops = [[0] * cols for _ in range(rows)], 0
    for i in range(rows):
        for j in range(cols):
            res = []
            for l, m in enumerate(ms):
                s = float(S[l][i, j])
                assert s == int(s)
                res.append(int(s) % m)
            out[i][j], o = garner(res, ms)
            ops += o
    return out, ops


def exact_product(X, Y):
    return [[sum(X[i][k] * Y[k][j] for k in range(len(Y))) for j in range(len(Y[0]))]
            for i in range(len(X))]


def test_residues_and_products_are_exact_in_bf16_and_fp32():
    """Symmetric residues of moduli up to 513 are at most 256 in magnitude,
    hence bf16-exact; K = 64 products of two of them stay below 2^22, so a
    float32 matmul in any order returns the exact integer sum."""
    for m in (256, 257, 511, 512, 513):
        assert all(bf16_exact(sym_res(x, m)) for x in range(m))
        assert max(abs(sym_res(x, m)) for x in range(m)) <= 256
    assert not bf16_exact(257)
    # worst case: every residue at the largest magnitude, same sign
    A = np.full((4, K), -256.0, dtype=np.float32)
    B = np.full((K, 4), -256.0, dtype=np.float32)
    assert (A @ B == K * 256 * 256).all() and K * 256 * 256 < 1 << 24
    # and a random matrix against integer arithmetic
    rng = np.random.default_rng(7)
    Ai = rng.integers(-256, 257, size=(16, K))
    Bi = rng.integers(-256, 257, size=(K, 16))
    assert ((Ai.astype(np.float32) @ Bi.astype(np.float32)).astype(np.int64) == Ai @ Bi).all()


def test_moduli_counts_against_scheme_one_pairs():
    """The modulus count scheme II needs on scheme I's 120-bit grid, with
    8-bit (INT8-style, <= 256) and bf16-exact (<= 513) moduli."""
    bits = product_bits(T_BITS, K)
    assert bits == 245
    m8 = moduli(256, bits)
    m9 = moduli(513, bits)
    assert len(m8) == 33
    assert len(m9) == 28
    for ms in (m8, m9):
        assert all(math.gcd(a, b) == 1 for i, a in enumerate(ms) for b in ms[i + 1:])
        assert math.prod(ms) >= 1 << bits
    # tensor work: one K = 64 product per modulus against one per digit pair
    assert SCHEME_I_PAIRS / len(m9) > 4.2
    # recombination per output entry: Garner's r (r - 1) / 2 modular
    # multiply-adds plus r - 1 wide multiply-adds, against scheme I's 15
    # shifted additions of exact diagonal sums
    r = len(m9)
    assert r * (r - 1) // 2 == 378
    assert (r * (r - 1) // 2 + r - 1) / SCHEME_I_DIAGONALS > 25


def test_scheme_two_recovers_exact_products():
    """Residue products + Garner give the exact integer product of random
    and extreme 120-bit operands (|X| < 2^119), K = 64, with the counted
    number of modular multiply-adds per entry."""
    bits = product_bits(T_BITS, K)
    ms = moduli(513, bits)
    rng = random.Random(2107)
    top = (1 << (T_BITS - 1)) - 1
    cases = [
        ([[rng.randint(-top, top) for _ in range(K)] for _ in range(3)],
         [[rng.randint(-top, top) for _ in range(4)] for _ in range(K)]),
        ([[top] * K for _ in range(2)], [[top] * 2 for _ in range(K)]),
        ([[-top] * K for _ in range(2)], [[top, -top] for _ in range(K)]),
        ([[rng.choice((-1, 1)) << rng.randint(0, T_BITS - 2) for _ in range(K)] for _ in range(2)],
         [[rng.choice((-1, 0, 1)) * rng.randint(0, top) for _ in range(3)] for _ in range(K)]),
    ]
    r = len(ms)
    for X, Y in cases:
        got, ops = scheme2_product(X, Y, ms)
        assert got == exact_product(X, Y)
        assert ops == len(X) * len(Y[0]) * r * (r - 1) // 2


def test_model_catches_a_missing_modulus():
    """With one modulus fewer the range no longer covers the extreme sums:
    the reconstruction of the all-maximal product goes wrong."""
    bits = product_bits(T_BITS, K)
    ms = moduli(513, bits)[:-1]
    assert math.prod(ms) < 1 << bits
    top = (1 << (T_BITS - 1)) - 1
    X = [[top] * K]
    Y = [[top] for _ in range(K)]
    got, _ = scheme2_product(X, Y, ms)
    assert got != exact_product(X, Y)
