"""The split-precision (Ozaki-style, bf16 tcgen05) trailing update for DD and
the standalone multiword GEMM (C -= A B, the paper's BNCmatmul block product,
Section 2), through the C ABI.

The plain GEMM is bitwise equal to the elimination's per-entry order.  The
split form is not bitwise: each 64-wide slab product is exact up to the
digit truncation and is rounded once, so its error is stated per result
against the exact product (error / (max_t|a_it| max_t|b_tj|) <= 2^-104 is
required; the bound of the method is 2^-107 plus the final DD rounding)."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import exact as X
from paper_2107_12550_gb300 import _lib as L
from paper_2107_12550_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2107_12550_gb300 import build as B
    B.build()


def api():
    from paper_2107_12550_gb300 import api as A
    return A


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _mat(w, rows, cols, seed, ld=None, scale_rows=False):
    g = np.random.default_rng(seed)
    ld = ld or rows + 3
    M = np.zeros((w, cols, ld))
    M[0, :, :rows] = g.uniform(-1, 1, (cols, rows))
    if scale_rows:
        M[0, :, :rows] *= np.ldexp(1.0, g.integers(-20, 20, rows))[None, :]
    for c in range(1, w):
        _, ex = np.frexp(M[c - 1, :, :rows])
        M[c, :, :rows] = np.where(M[c - 1, :, :rows] == 0, 0.0,
                                  np.ldexp(g.uniform(-1, 1, (cols, rows)), ex - 55))
    return M


@pytest.mark.parametrize("tile", [0, 1, 2, 3])
@pytest.mark.parametrize("w", [2, 3, 4])
def test_gemm_sub_plain_bitwise(w, tile):
    """Every tile variant of the plain update (MW_TUNE_GEMM_TILE: 0 automatic,
    1-3 forced) gives the oracle's operation sequence bitwise; 70 x 45 leaves
    a ragged tail for every tile size and K = 21 a ragged K chunk."""
    m, N, K = 70, 45, 21
    C = _mat(w, m, N, 1)
    A = _mat(w, m, K, 2)
    B = _mat(w, K, N, 3)
    lib = L.lib()
    prev = lib.mw_set_tuning(L.MW_TUNE_GEMM_TILE, w, tile)
    assert prev >= 0
    try:
        got = host(api().gemm_sub(dev(C), dev(A), dev(B), m, w, "plain"))
    finally:
        lib.mw_set_tuning(L.MW_TUNE_GEMM_TILE, w, prev)
    ref = C[:, :, :m].copy()
    for t in range(K):
        a = np.repeat(A[:, t, :m][:, None, :], N, axis=1).reshape(w, -1)      # (w, N*m)
        b = np.repeat(B[:, :, t][:, :, None], m, axis=2).reshape(w, -1)
        prod = oracle.arith(oracle.OP_MUL, w, a, b)
        ref = oracle.arith(oracle.OP_SUB, w, ref.reshape(w, -1), prod).reshape(w, N, m)
    assert np.array_equal(got[:, :, :m], ref)


@pytest.mark.parametrize("tile", [0, 1, 3])
@pytest.mark.parametrize("w", [2, 3, 4])
def test_gemm_add_plain_bitwise(w, tile):
    """C += A B (the standalone block matrix product) on every tile variant:
    each entry applies c = c + a_t b_t in ascending t with the oracle's
    multiword multiply and add, bitwise; gemm() from a zero C likewise."""
    m, N, K = 70, 45, 21
    C = _mat(w, m, N, 31)
    A = _mat(w, m, K, 32)
    B = _mat(w, K, N, 33)
    lib = L.lib()
    prev = lib.mw_set_tuning(L.MW_TUNE_GEMM_TILE, w, tile)
    try:
        got = host(api().gemm_add(dev(C), dev(A), dev(B), m, w, "plain"))
        got0 = host(api().gemm(dev(A), dev(B), m, w, "plain"))
    finally:
        lib.mw_set_tuning(L.MW_TUNE_GEMM_TILE, w, prev)
    for start, res in ((C[:, :, :m].copy(), got), (np.zeros((w, N, m)), got0)):
        ref = start
        for t in range(K):
            a = np.repeat(A[:, t, :m][:, None, :], N, axis=1).reshape(w, -1)
            b = np.repeat(B[:, :, t][:, :, None], m, axis=2).reshape(w, -1)
            prod = oracle.arith(oracle.OP_MUL, w, a, b)
            ref = oracle.arith(oracle.OP_ADD, w, ref.reshape(w, -1), prod).reshape(w, N, m)
        assert np.array_equal(res[:, :, :m], ref)


@pytest.mark.parametrize("update", ["plain", "split"])
def test_gemm_add_is_negated_sub(update):
    """Multiword addition and the greedy rounding are odd functions, so
    C + A B = -((-C) - A B) bitwise, for both update forms."""
    m, N, K = 150, 40, 128
    C = _mat(2, m, N, 41)
    A = _mat(2, m, K, 42)
    B = _mat(2, K, N, 43)
    ga = host(api().gemm_add(dev(C), dev(A), dev(B), m, 2, update))
    gs = host(api().gemm_sub(dev(-C), dev(A), dev(B), m, 2, update))
    assert np.array_equal(ga[:, :, :m], -gs[:, :, :m])


def test_gemm_add_split_error_per_result():
    """Split C += A B: per result, |C_out - (C + A B)| minus the final DD
    rounding is at most 2^-104 max|a| max|b| (exact products from the oracle)."""
    m, N, K = 130, 70, 64
    C = _mat(2, m, N, 51)
    A = _mat(2, m, K, 52, scale_rows=True)
    B = _mat(2, K, N, 53)
    got = host(api().gemm_add(dev(C), dev(A), dev(B), m, 2, "split"))
    worst = 0.0
    for i in range(0, m, 3):
        amax = np.max(np.abs(A[0, :, i]))
        for j in range(0, N, 2):
            bmax = np.max(np.abs(B[0, j, :K]))
            xs = np.concatenate([A[0, :, i], A[0, :, i], A[1, :, i], A[1, :, i]])
            ys = np.concatenate([B[0, j, :K], B[1, j, :K], B[0, j, :K], B[1, j, :K]])
            P = oracle.exact_dot(xs, ys, 4)
            exact = X.words_to_frac(C[:, j, i]) + X.words_to_frac(P)
            err = abs(X.words_to_frac(got[:, j, i]) - exact)
            allowed_rounding = Fraction(3, 2 ** 106) * abs(exact)
            ratio = max(err - allowed_rounding, Fraction(0)) / (Fraction(amax) * Fraction(bmax))
            worst = max(worst, float(ratio))
    assert worst <= 2.0 ** -104


@pytest.mark.parametrize("m,N,scaled", [(130, 70, False), (257, 33, True), (64, 32, False)])
def test_gemm_sub_split_error_per_result(m, N, scaled):
    K = 64
    C = _mat(2, m, N, 11)
    A = _mat(2, m, K, 12, scale_rows=scaled)
    B = _mat(2, K, N, 13)
    got = host(api().gemm_sub(dev(C), dev(A), dev(B), m, 2, "split"))
    worst = 0.0
    for i in range(0, m, 3):
        amax = np.max(np.abs(A[0, :, i]))
        for j in range(0, N, 2):
            bmax = np.max(np.abs(B[0, j, :K]))
            xs = np.concatenate([A[0, :, i], A[0, :, i], A[1, :, i], A[1, :, i]])
            ys = np.concatenate([B[0, j, :K], B[1, j, :K], B[0, j, :K], B[1, j, :K]])
            P = oracle.exact_dot(xs, ys, 4)
            exact = X.words_to_frac(C[:, j, i]) - X.words_to_frac(P)
            err = abs(X.words_to_frac(got[:, j, i]) - exact)
            # the final DD rounding of the result is allowed on top
            allowed_rounding = Fraction(3, 2 ** 106) * abs(exact)
            ratio = max(err - allowed_rounding, Fraction(0)) / (Fraction(amax) * Fraction(bmax))
            worst = max(worst, float(ratio))
    print(f"split GEMM m={m} N={N}: max |dC|/(max|a| max|b|) = 2^{math.log2(worst) if worst else -math.inf:.1f}")
    assert worst <= 2.0 ** -104


def test_gemm_sub_split_matches_plain_closely():
    m, N, K = 300, 200, 128
    C = _mat(2, m, N, 21)
    A = _mat(2, m, K, 22)
    B = _mat(2, K, N, 23)
    gs = host(api().gemm_sub(dev(C), dev(A), dev(B), m, 2, "split"))
    gp = host(api().gemm_sub(dev(C), dev(A), dev(B), m, 2, "plain"))
    d = np.abs((gs[0, :, :m] - gp[0, :, :m]) + (gs[1, :, :m] - gp[1, :, :m]))
    assert d.max() <= 2.0 ** -95 * K


def _eta(s_A, s_b, x):
    n = x.shape[1]
    r = oracle.residual(s_A, s_b, x, 8)
    Ainf = np.max(np.sum(np.abs(s_A[0, :, :n]), axis=0))
    return np.max(np.abs(r[0])) / (Ainf * np.max(np.abs(x[0])) + np.max(np.abs(s_b[0])))


@pytest.mark.parametrize("n", [65, 200, 300, 513])
def test_lu_split_backward_error_and_pivots(n):
    s = W.uniform_system(n, words=2, seed=40 + n, b_words=2)
    A = dev(s.A)
    LUs, pivs, infos = api().ludecomp(A, 2, "split")
    LUp, pivp, infop = api().ludecomp(A, 2, "plain")
    xs = host(api().solve(LUs, pivs, dev(s.b), 2))
    eta = _eta(s.A, s.b, xs)
    assert eta <= 1e-28, eta
    diff = int((host(pivs) != host(pivp)).sum())
    print(f"n={n}: split-vs-plain pivot differences {diff}, eta {eta:.2e}")
    assert diff <= n // 50


def test_lu_split_full_size_backward_error():
    """n = 4096 DD (the large-LU configuration), split trailing update:
    normwise backward error of the solution <= 1e-28 (exact CPU residual)."""
    s = W.uniform_system(4096, words=2, seed=0, b_words=2)
    LU, piv, info = api().ludecomp(dev(s.A), 2, "split")
    assert int(info.item()) == 0
    x = host(api().solve(LU, piv, dev(s.b), 2))
    eta = _eta(s.A, s.b, x)
    print(f"n=4096 split: eta {eta:.2e}")
    assert eta <= 1e-28


def _first_columns_bitwise(A, w, LUg, pivg, ks=8):
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


@pytest.mark.parametrize("n", [4096, 8192])
def test_config3_full_size_plain_and_split(n):
    """The large-LU configuration at full size, n = 4096 and 8192 DD (uniform
    entries): the plain LU's pivots and first 8 columns bitwise equal to the
    oracle's first 8 steps (sampled), the split LU's normwise backward error
    <= 1e-28 (exact residual) with pivots equal to the plain LU's up to
    near-ties."""
    s = W.uniform_system(n, words=2, seed=0, b_words=2)
    A = dev(s.A)
    LUp, pivp, infop = api().ludecomp(A, 2, "plain")
    assert int(infop.item()) == 0
    pivp = host(pivp)
    _first_columns_bitwise(s.A, 2, host(LUp), pivp)
    del LUp
    LUs, pivs, infos = api().ludecomp(A, 2, "split")
    assert int(infos.item()) == 0
    x = host(api().solve(LUs, pivs, dev(s.b), 2))
    eta = _eta(s.A, s.b, x)
    diff = int((host(pivs) != pivp).sum())
    print(f"n={n} split: eta {eta:.2e}, pivots differing from plain {diff}")
    assert eta <= 1e-28
    assert diff <= n // 50


def test_config2_n2048_td_lu_first_columns_bitwise():
    """The bench's TD LU at n = 2048 (SVD-built, kappa 2^33), full size:
    pivots and the first 8 columns bitwise equal to the oracle's first 8
    elimination steps, with the GPU's later row swaps applied."""
    s = W.svd_system(2048, 10.0, seed=0)
    A3 = np.ascontiguousarray(s.A[:3])
    LU, piv, info = api().ludecomp(dev(A3), 3)
    assert int(info.item()) == 0
    _first_columns_bitwise(A3, 3, host(LU), host(piv))


def test_refine_split_dd_inner():
    s = W.svd_system(300, 10.0, seed=7)
    res = api().refine(dev(s.A), dev(s.b), 2, 200, update="split")
    assert res.status == 0
    x = host(res.x)
    for i in range(0, 300, 5):
        assert abs(X.words_to_frac(x[:, i]) - 1) <= Fraction(1, 2 ** 200)


@pytest.mark.parametrize("leaf", [8, 16, 32])
def test_lu_split_recursive_panel(leaf):
    """The split LU of one system with its panels factored recursively down
    to `leaf` columns (MW_TUNE_SPLIT_PANEL_LEAF): backward error <= 1e-28 and
    pivots as the oracle's up to near-ties."""
    from paper_2107_12550_gb300 import _lib as L
    lib = L.lib()
    prev = lib.mw_set_tuning(L.MW_TUNE_SPLIT_PANEL_LEAF, 2, leaf)
    try:
        for n in (200, 513):
            s = W.uniform_system(n, words=2, seed=60 + n, b_words=2)
            LUs, pivs, info = api().ludecomp(dev(s.A), 2, "split")
            assert int(info.item()) == 0
            xs = host(api().solve(LUs, pivs, dev(s.b), 2))
            eta = _eta(s.A, s.b, xs)
            assert eta <= 1e-28, (n, eta)
            _, pivo, _ = oracle.lu(2, s.A)
            assert int((host(pivs) != pivo).sum()) <= n // 50
    finally:
        lib.mw_set_tuning(L.MW_TUNE_SPLIT_PANEL_LEAF, 2, prev)
