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
from parity_rules import check_pivots_near_tie, eta as _eta, exact_solution, first_columns_bitwise, forward_error

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


def _split_errors(C, A, B, got, m, N, K, sign):
    """Per result (every entry): the error of the split product against
    the exact C + sign A B, less the final DD rounding, normalised two ways:
    by max_t|a_it| max_t|b_tj| (the method's a-priori bound, 2^-107 per slab)
    and by (|A| |B|)_ij (the elementwise measure, stated per result)."""
    absAB = np.abs(A[0, :, :m]).T @ np.abs(B[0, :, :K]).T      # (m, N)
    worst_max = worst_el = 0.0
    for i in range(m):
        amax = np.max(np.abs(A[0, :, i]))
        for j in range(N):
            bmax = np.max(np.abs(B[0, j, :K]))
            xs = np.concatenate([A[0, :, i], A[0, :, i], A[1, :, i], A[1, :, i]])
            ys = np.concatenate([B[0, j, :K], B[1, j, :K], B[0, j, :K], B[1, j, :K]])
            P = oracle.exact_dot(xs, ys, 4)
            exact = X.words_to_frac(C[:, j, i]) + sign * X.words_to_frac(P)
            err = abs(X.words_to_frac(got[:, j, i]) - exact)
            allowed_rounding = Fraction(3, 2 ** 106) * abs(exact)
            e = max(err - allowed_rounding, Fraction(0))
            if e:
                worst_max = max(worst_max, float(e / (Fraction(amax) * Fraction(bmax))))
                worst_el = max(worst_el, float(e / Fraction(absAB[i, j])))
    return worst_max, worst_el


def _lg(v):
    return math.log2(v) if v else -math.inf


def test_gemm_add_split_error_per_result():
    """Split C += A B: per result, |C_out - (C + A B)| minus the final DD
    rounding is at most 2^-104 max|a| max|b| (exact products from the oracle)."""
    m, N, K = 130, 70, 64
    C = _mat(2, m, N, 51)
    A = _mat(2, m, K, 52, scale_rows=True)
    B = _mat(2, K, N, 53)
    got = host(api().gemm_add(dev(C), dev(A), dev(B), m, 2, "split"))
    worst, worst_el = _split_errors(C, A, B, got, m, N, K, +1)
    print(f"split C += AB: per result 2^{_lg(worst):.1f} of max|a|max|b|, 2^{_lg(worst_el):.1f} of (|A||B|)_ij")
    assert worst <= 2.0 ** -104
    assert worst_el <= 2.0 ** -100


@pytest.mark.parametrize("m,N,scaled", [(130, 70, False), (257, 33, True), (64, 32, False)])
def test_gemm_sub_split_error_per_result(m, N, scaled):
    K = 64
    C = _mat(2, m, N, 11)
    A = _mat(2, m, K, 12, scale_rows=scaled)
    B = _mat(2, K, N, 13)
    got = host(api().gemm_sub(dev(C), dev(A), dev(B), m, 2, "split"))
    worst, worst_el = _split_errors(C, A, B, got, m, N, K, -1)
    print(f"split GEMM m={m} N={N}: max |dC|/(max|a| max|b|) = 2^{_lg(worst):.1f}, "
          f"max |dC|/(|A||B|)_ij = 2^{_lg(worst_el):.1f}")
    assert worst <= 2.0 ** -104
    assert worst_el <= 2.0 ** -100


@pytest.mark.parametrize("m,N,plus,scaled,off_grid", [(130, 70, False, False, False), (257, 33, True, True, False),
                                                       (64, 48, False, False, True), (129, 17, True, False, True)])
def test_split_slab_bitwise_against_model(m, N, plus, scaled, off_grid):
    """One 64-wide slab of the split product, C -= A B (plus: C += A B),
    bitwise against the oracle's statement of the method (oracle/ozaki.py:
    scales, floored integers, 15 balanced digits, pairs p + q <= 16, the
    exact form C -/+ P rounded once, else the rounded product and the DD
    subtraction).  Ragged tiles in both directions; rows scaled by 2^+-20;
    with off_grid, a third of C is far below the product's grid, so those
    entries take the second form.  Bit patterns are compared, signs of
    zeros included."""
    from oracle import ozaki as Z
    K = 64
    C = _mat(2, m, N, 61)
    A = _mat(2, m, K, 62, scale_rows=scaled)
    B = _mat(2, K, N, 63)
    if off_grid:
        g = np.random.default_rng(64)
        pick = g.random((N, m)) < 1 / 3
        C[0, :, :m] = np.where(pick, C[0, :, :m] * 2.0 ** -200, C[0, :, :m])
        C[1, :, :m] = np.where(pick, C[1, :, :m] * 2.0 ** -200, C[1, :, :m])
    fn = api().gemm_add if plus else api().gemm_sub
    got = host(fn(dev(C), dev(A), dev(B), m, 2, "split"))
    ref, nexact = Z.update(C, A, B, m, N, K, plus=plus)
    print(f"m={m} N={N}: {nexact} of {m * N} entries in the exact form")
    if off_grid:
        assert nexact < m * N          # some entries take the rounded-product form
    assert np.array_equal(got[:, :, :m].view(np.int64), ref.view(np.int64))


def test_gemm_sub_split_matches_plain_closely():
    m, N, K = 300, 200, 128
    C = _mat(2, m, N, 21)
    A = _mat(2, m, K, 22)
    B = _mat(2, K, N, 23)
    gs = host(api().gemm_sub(dev(C), dev(A), dev(B), m, 2, "split"))
    gp = host(api().gemm_sub(dev(C), dev(A), dev(B), m, 2, "plain"))
    d = np.abs((gs[0, :, :m] - gp[0, :, :m]) + (gs[1, :, :m] - gp[1, :, :m]))
    assert d.max() <= 2.0 ** -95 * K


@pytest.mark.parametrize("n", [65, 200, 300, 513])
def test_lu_split_backward_error_and_pivots(n):
    """Split LU of one DD system: pivots as the oracle's up to a near-tie,
    eta <= 1e-28 (exact residual), and the forward error within 10x the
    oracle's own DD direct solve."""
    s = W.uniform_system(n, words=2, seed=40 + n, b_words=2)
    A = dev(s.A)
    LUs, pivs, infos = api().ludecomp(A, 2, "split")
    xs = host(api().solve(LUs, pivs, dev(s.b), 2))
    e = _eta(s.A, s.b, xs)
    assert e <= 1e-28, e
    LUo, pivo, _ = oracle.lu(2, s.A)
    k = check_pivots_near_tie(s.A, 2, host(pivs), pivo)
    xo = oracle.solve(2, LUo, pivo, s.b)
    xstar = exact_solution(s.A, s.b)
    fe_gpu, fe_orc = forward_error(xs, xstar), forward_error(xo, xstar)
    print(f"n={n}: first pivot divergence {k}, eta {e:.2e}, forward error {float(fe_gpu):.2e} "
          f"(oracle {float(fe_orc):.2e})")
    assert fe_gpu <= 10 * fe_orc


def test_lu_split_full_size_backward_error():
    """n = 4096 DD (the large-LU configuration), split trailing update:
    normwise backward error of the solution <= 1e-28 (exact CPU residual)."""
    s = W.uniform_system(4096, words=2, seed=0, b_words=2)
    LU, piv, info = api().ludecomp(dev(s.A), 2, "split")
    assert int(info.item()) == 0
    x = host(api().solve(LU, piv, dev(s.b), 2))
    e = _eta(s.A, s.b, x)
    print(f"n=4096 split: eta {e:.2e}")
    assert e <= 1e-28


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
    first_columns_bitwise(s.A, 2, host(LUp), pivp)
    del LUp
    LUs, pivs, infos = api().ludecomp(A, 2, "split")
    assert int(infos.item()) == 0
    x = host(api().solve(LUs, pivs, dev(s.b), 2))
    e = _eta(s.A, s.b, x)
    k = check_pivots_near_tie(s.A, 2, host(pivs), pivp)
    print(f"n={n} split: eta {e:.2e}, first pivot divergence from the plain path {k}")
    assert e <= 1e-28


def test_config2_n2048_qd_lu_first_columns_and_backward_error():
    """Config 2's QD LU + solve at n = 2048 (SVD-built, kappa 2^33), full
    size: pivots and the first 8 columns bitwise equal to the oracle's first
    8 elimination steps (with the GPU's later row swaps applied), and the
    direct QD solve's normwise backward error <= 1e-60 by an exact residual."""
    s = W.svd_system(2048, 10.0, seed=0)
    LU, piv, info = api().ludecomp(dev(s.A), 4)
    assert int(info.item()) == 0
    pv = host(piv)
    first_columns_bitwise(s.A, 4, host(LU), pv)
    x = host(api().solve(LU, piv, dev(s.b), 4))
    e = _eta(s.A, s.b, x)
    print(f"n=2048 QD direct: eta {e:.2e}")
    assert e <= 1e-60


def test_config2_n2048_td_lu_first_columns_bitwise():
    """The bench's TD LU at n = 2048 (SVD-built, kappa 2^33), full size:
    pivots and the first 8 columns bitwise equal to the oracle's first 8
    elimination steps, with the GPU's later row swaps applied."""
    s = W.svd_system(2048, 10.0, seed=0)
    A3 = np.ascontiguousarray(s.A[:3])
    LU, piv, info = api().ludecomp(dev(A3), 3)
    assert int(info.item()) == 0
    first_columns_bitwise(A3, 3, host(LU), host(piv))


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
            e = _eta(s.A, s.b, xs)
            assert e <= 1e-28, (n, e)
            _, pivo, _ = oracle.lu(2, s.A)
            check_pivots_near_tie(s.A, 2, host(pivs), pivo)
    finally:
        lib.mw_set_tuning(L.MW_TUNE_SPLIT_PANEL_LEAF, 2, prev)


@pytest.mark.parametrize("update,w,n,leaf", [("plain", 2, 300, 0), ("plain", 3, 700, 0), ("plain", 4, 257, 0),
                                             ("split", 2, 1000, 0), ("split", 2, 1000, 16),
                                             ("split", 2, 2048, 32)])
def test_lu_lookahead_bitwise_equal_to_serial(update, w, n, leaf):
    """The blocked look-ahead (MW_TUNE_LOOKAHEAD: the next panel factored on
    a second stream while the rest of the trailing matrix is updated) gives
    the serial schedule's factors and pivots bit for bit: every entry gets the
    same operations in the same order.  Ragged last panels included."""
    lib = L.lib()
    s = W.uniform_system(n, words=w, seed=70 + n, b_words=w)
    prev_la = lib.mw_get_tuning(L.MW_TUNE_LOOKAHEAD, w)
    prev_leaf = lib.mw_get_tuning(L.MW_TUNE_SPLIT_PANEL_LEAF, 2)
    out = {}
    try:
        lib.mw_set_tuning(L.MW_TUNE_SPLIT_PANEL_LEAF, 2, leaf)
        for la in (0, 1, 1):
            lib.mw_set_tuning(L.MW_TUNE_LOOKAHEAD, w, la)
            LU, piv, info = api().ludecomp(dev(s.A), w, update)
            out.setdefault(la, []).append((host(LU), host(piv), int(info.item())))
    finally:
        lib.mw_set_tuning(L.MW_TUNE_LOOKAHEAD, w, prev_la)
        lib.mw_set_tuning(L.MW_TUNE_SPLIT_PANEL_LEAF, 2, prev_leaf)
    ref = out[0][0]
    for LU, piv, info in out[1]:
        assert info == ref[2]
        assert np.array_equal(piv, ref[1])
        assert np.array_equal(LU.view(np.uint64), ref[0].view(np.uint64))
