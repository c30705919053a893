"""GPU parity: every call goes through the C ABI (libmwlu.so) and is compared
with the CPU oracle on the same seeded inputs.  The plain path is required to
be bitwise identical (same algorithms, same per-element operation order);
the exact residual is identical by construction (exact, then greedy
round-to-nearest)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import exact as X
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


def _rand_mw(rng, w, cnt, cancel=False):
    e = rng.integers(-30, 30, cnt)
    x = np.zeros((w, cnt))
    x[0] = np.ldexp(rng.uniform(-1, 1, cnt), e)
    for c in range(1, w):
        _, ex = np.frexp(x[c - 1])
        x[c] = np.where(x[c - 1] == 0, 0.0, np.ldexp(rng.uniform(-1, 1, cnt), ex - 55))
    if cancel:
        y = -x.copy()
        y[w - 1] = y[w - 1] * (1 + rng.uniform(-1e-3, 1e-3, cnt))
        return x, y
    return x


@pytest.mark.parametrize("w", [2, 3, 4])
def test_arith_bitwise(w):
    rng = np.random.default_rng(5 + w)
    cnt = 20000
    x = _rand_mw(rng, w, cnt)
    y = _rand_mw(rng, w, cnt)
    xc, yc = _rand_mw(rng, w, 2000, cancel=True)
    x = np.concatenate([x, xc], axis=1)
    y = np.concatenate([y, yc], axis=1)
    y[:, :50] = x[:, :50]            # exact ties for the comparison
    y[0, 50:60] = 0.0                # zero leading words
    y[:, 60:70] = 0.0
    y[0, 60:70] = 1.0
    for op in range(5):
        got = host(api().arith(op, w, dev(x), dev(y)))
        ref = oracle.arith(op, w, x, y)
        if op == 4:
            assert np.array_equal(got[0].astype(np.int64), ref)
        else:
            assert np.array_equal(got, ref, equal_nan=True), (op, np.argwhere(got != ref)[:5])


def _twosum_edge_inputs(rng, w, cnt):
    """Pairs aimed at every branch of the integer TwoSum: leading-word
    exponent gaps 0..70 (the s = a, e = b cut at a gap of 55), exact and
    near cancellation, halfway cases (ties to even, also below a power of
    two), zeros of both signs, subnormals, and sums near overflow."""
    x = _rand_mw(rng, w, cnt)
    y = _rand_mw(rng, w, cnt)
    q = cnt // 8
    k = np.arange(cnt)
    gap = rng.integers(0, 71, cnt)
    sel = k < q                                               # exponent gaps
    y[0, sel] = np.ldexp(rng.uniform(0.5, 1.0, q) * rng.choice([-1.0, 1.0], q), np.frexp(x[0, sel])[1] - gap[sel])
    sel = (k >= q) & (k < 2 * q)                              # exact cancellation in any word
    y[:, sel] = -x[:, sel]
    sel = (k >= 2 * q) & (k < 3 * q)                          # a few ulps apart, opposite signs
    y[0, sel] = -np.nextafter(x[0, sel], np.where(rng.random(q) < 0.5, np.inf, -np.inf))
    sel = (k >= 3 * q) & (k < 4 * q)                          # halfway: y0 = +-ulp(x0) / 2 (+ tail)
    ulp = np.spacing(np.abs(x[0, sel]))
    y[0, sel] = ulp / 2 * rng.choice([-1.0, 1.0], q)
    y[1:, sel] = 0.0
    sel = (k >= 4 * q) & (k < 5 * q)                          # powers of two minus tiny values
    x[0, sel] = np.ldexp(1.0, rng.integers(-20, 20, q)) * rng.choice([-1.0, 1.0], q)
    y[0, sel] = -np.sign(x[0, sel]) * np.spacing(np.abs(x[0, sel])) * rng.choice([0.25, 0.5, 0.75, 1.0], q)
    sel = (k >= 5 * q) & (k < 6 * q)                          # signed zeros anywhere
    z = rng.choice([0.0, -0.0], (w, q))
    m = rng.random((w, q)) < 0.5
    y[:, sel] = np.where(m, z, y[:, sel])
    sel = (k >= 6 * q) & (k < 7 * q)                          # subnormal and tiny words
    x[:, sel] = rng.choice([5e-324, -5e-324, 2.2250738585072014e-308, -1.1e-308, 3e-310], (w, q))
    y[:, sel] = rng.choice([5e-324, -2.2250738585072014e-308, 1e-309, -4e-323], (w, q))
    sel = k >= 7 * q                                          # near overflow
    r = cnt - 7 * q
    x[0, sel] = rng.choice([1.7e308, -1.7e308, 8.9e307], r)
    y[0, sel] = rng.choice([1.7e308, 8.98846567431158e307, -1.0], r)
    x[1:, sel] = 0.0
    y[1:, sel] = 0.0
    return x, y


@pytest.mark.parametrize("w", [2, 3, 4])
def test_arith_twosum_edge_cases(w):
    """Addition, multiplication and division on inputs aimed at the integer
    TwoSum's branches and fallbacks: every result bitwise equal to the
    oracle's FP64 TwoSum arithmetic (NaNs compared as NaNs)."""
    rng = np.random.default_rng(91 + w)
    x, y = _twosum_edge_inputs(rng, w, 16000)
    for op in range(4):
        got = host(api().arith(op, w, dev(x), dev(y)))
        ref = oracle.arith(op, w, x, y)
        same_bits = (got.view(np.uint64) == ref.view(np.uint64)) | (np.isnan(got) & np.isnan(ref))
        assert same_bits.all(), (op, np.argwhere(~same_bits)[:5])


@pytest.mark.parametrize("w", [2, 3, 4])
def test_cmpabs_special_values(w):
    """The magnitude comparison of the pivot search on signed zeros,
    infinities, NaNs, subnormals and ties in every word, against the
    oracle's floating-point comparison (a NaN word pair is unordered)."""
    special = np.array([0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, np.nan, -np.nan, 5e-324, -5e-324,
                        2.2250738585072014e-308, -1.5, 1.5, 3.0, -3.0, 1e300, -1e-300])
    rng = np.random.default_rng(71 + w)
    cnt = 6000
    x = special[rng.integers(0, len(special), (w, cnt))]
    y = special[rng.integers(0, len(special), (w, cnt))]
    y[:, :500] = x[:, :500]
    y[0, 500:1500] = x[0, 500:1500]                  # equal leading words, later words decide
    y[0, 1500:2000] = -x[0, 1500:2000]               # opposite signs of the same magnitude
    got = host(api().arith(4, w, dev(x), dev(y)))
    ref = oracle.arith(oracle.OP_CMPABS, w, x, y)
    assert np.array_equal(got[0].astype(np.int64), ref), np.argwhere(got[0].astype(np.int64) != ref)[:5]


def _lu_compare(A, w, update="plain"):
    LUg, pivg, infog = api().ludecomp(dev(A), w, update)
    LUo, pivo, infoo = oracle.lu(w, A)
    LUg = host(LUg)
    n = A.shape[1]
    assert int(host(infog)[0]) == infoo
    assert np.array_equal(host(pivg), pivo)
    assert np.array_equal(LUg[:, :, :n], LUo[:, :, :n])
    return LUo, pivo


@pytest.mark.parametrize("w", [2, 3, 4])
@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 63, 64, 65, 100, 129, 200])
def test_lu_bitwise(w, n):
    A = W.uniform_matrix(n, w, seed=1000 + 7 * n + w)
    _lu_compare(A, w)


@pytest.mark.parametrize("w", [2, 3, 4])
def test_lu_bitwise_odd_lda_and_svd(w):
    A = W.uniform_matrix(150, w, seed=3, lda=157)
    _lu_compare(A, w)
    s = W.svd_system(130, 12.0, seed=4)
    _lu_compare(s.A[:w].copy(), w)


@pytest.mark.parametrize("w", [2, 3, 4])
def test_lu_singular_and_degenerate(w):
    n = 70
    A = np.zeros((w, n, n))
    rng = np.random.default_rng(9)
    A[0] = rng.integers(-5, 6, (n, n)).astype(float)
    A[0, 40] = 0.0                    # zero column 40 -> a zero pivot at some step
    A[0, 41] = 2 * A[0, 3]            # dependent columns
    _lu_compare(A, w)
    Z = np.zeros((w, 33, 33))
    _lu_compare(Z, w)
    P = np.zeros((w, 97, 97))
    perm = rng.permutation(97)
    for i in range(97):
        P[0, perm[i], i] = 1.0
    _lu_compare(P, w)


def test_lu_empty():
    A = torch.zeros((2, 0, 1), dtype=torch.float64, device="cuda")
    LU, piv, info = api().ludecomp(A, 2)
    assert int(info.item()) == 0


@pytest.mark.parametrize("w", [2, 3, 4])
@pytest.mark.parametrize("n", [1, 33, 100, 257])
def test_solve_bitwise(w, n):
    A = W.uniform_matrix(n, w, seed=77 + n)
    LUo, pivo, info = oracle.lu(w, A)
    b = _rand_mw(np.random.default_rng(n), w, n)
    xg = host(api().solve(dev(LUo), torch.from_numpy(pivo).cuda(), dev(b), w))
    xo = oracle.solve(w, LUo, pivo, b)
    assert np.array_equal(xg, xo)
    # b aliased with x
    bt = dev(b)
    api().solve(dev(LUo), torch.from_numpy(pivo).cuda(), bt, w, out=bt)
    assert np.array_equal(host(bt), xo)


@pytest.mark.parametrize("n,wa,wb,wx,wr", [(1, 1, 1, 1, 1), (37, 2, 2, 8, 8), (100, 4, 8, 8, 8),
                                           (65, 3, 1, 5, 4), (300, 4, 8, 8, 8)])
def test_residual_bitwise(n, wa, wb, wx, wr):
    rng = np.random.default_rng(n + wa)
    A = np.zeros((wa, n, n + 3))
    for c in range(wa):
        A[c, :, :n] = np.ldexp(rng.uniform(-1, 1, (n, n)), -54 * c + rng.integers(-3, 3))
    x = np.stack([np.ldexp(rng.uniform(-1, 1, n), -53 * d + 5) for d in range(wx)])
    b = np.stack([np.ldexp(rng.uniform(-1, 1, n), -53 * d) for d in range(wb)])
    if n > 10:
        x[:, 3] = 0.0
        A[:, 2, :] = 0.0
        b[0, 4] = 2.0 ** -1074          # subnormal terms
        A[0, 5, 6] = 2.0 ** -1070
        x[0, 5] = 2.0 ** -1000
    got = host(api().residual(dev(A), dev(b), dev(x), wr))
    ref = oracle.residual(A, b, x, wr)
    assert np.array_equal(got, ref)


def test_residual_matches_fraction_small():
    rng = np.random.default_rng(3)
    n = 6
    A = np.zeros((2, n, n))
    A[0] = rng.uniform(-1, 1, (n, n))
    A[1] = A[0] * 2.0 ** -60
    x = np.zeros((3, n))
    x[0] = rng.uniform(-1, 1, n)
    x[2] = x[0] * 2.0 ** -130
    b = np.zeros((1, n))
    b[0] = rng.uniform(-1, 1, n)
    got = host(api().residual(dev(A), dev(b), dev(x), 8))
    rf = X.residual(X.mat_to_frac(A, n), X.vec_to_frac(b), X.vec_to_frac(x))
    for i in range(n):
        assert list(got[:, i]) == X.greedy_words(rf[i], 8)


@pytest.mark.parametrize("w_in", [2, 3, 4])
@pytest.mark.parametrize("stop_mode", [0, 1])
def test_refine_bitwise(w_in, stop_mode):
    s = W.svd_system(90, 10.0, seed=21)
    res = api().refine(dev(s.A), dev(s.b), w_in, 200, stop_mode=stop_mode, rtol=1e-90)
    st, xo, corr, nres, info = oracle.refine(s.A, s.b, w_in, stop_mode=stop_mode, rtol=1e-90)
    assert res.status == st
    assert (res.corrections, res.residuals, res.info) == (corr, nres, info)
    assert np.array_equal(host(res.x), xo)
    assert X.forward_error(X.vec_to_frac(xo), [Fraction(1)] * 90) <= Fraction(1, 2 ** 200)


def test_refine_dd_rhs_and_limits():
    s = W.uniform_system(70, words=2, seed=12, b_words=2)
    res = api().refine(dev(s.A), dev(s.b), 2, 200)
    st, xo, corr, nres, info = oracle.refine(s.A, s.b, 2)
    assert res.status == st == 0 and np.array_equal(host(res.x), xo)
    res = api().refine(dev(s.A), dev(s.b), 2, 200, max_iter=0)
    assert res.status == 2 and res.corrections == 0 and res.residuals == 1
    Z = np.zeros((2, 8, 8))
    res = api().refine(dev(Z), dev(np.ones((2, 8))), 2, 200)
    assert res.status == 1 and res.info == 1


@pytest.mark.parametrize("w,u,y", [(2, 35, 105), (3, 45, 45), (4, 35, 105)])
def test_back_substitution_reciprocal_case(w, u, y):
    """The oracle pin that separates the two readings of the back
    substitution (y/u is an integer; y * RN(1/u) is not): the GPU solve
    gives the oracle's value, bitwise."""
    A = np.zeros((w, 1, 1)); A[0, 0, 0] = float(u)
    b = np.zeros((w, 1)); b[0, 0] = float(y)
    LU, piv, info = api().ludecomp(dev(A), w)
    xg = host(api().solve(LU, piv, dev(b), w))
    LUo, pivo, _ = oracle.lu(w, A)
    xo = oracle.solve(w, LUo, pivo, b)
    assert np.array_equal(xg, xo)
    assert X.words_to_frac(xg[:, 0]) != Fraction(y, u)


def test_refine_stagnation_exit_case():
    """The oracle's hand-traced stagnation case (A = 1/4 in four words whose
    DD part is 1, b = 1): the GPU refinement stops after 2 corrections as
    not converged, with x = 37/16, as the oracle does."""
    A = np.zeros((4, 1, 1)); A[0, 0, 0] = 1.0; A[2, 0, 0] = -0.75
    b = np.ones((1, 1))
    res = api().refine(dev(A), dev(b), 2, 200)
    st, xo, corr, nres, info = oracle.refine(A, b, 2)
    assert (res.status, res.corrections, res.residuals) == (st, corr, nres) == (2, 2, 2)
    assert np.array_equal(host(res.x), xo)


def test_config1_dd_n256_bitwise():
    """Single DD LU + substitution at n = 256 (uniform entries, b = A*1
    rounded to DD), plain path: bitwise equal to the oracle."""
    s = W.uniform_system(256, words=2, seed=0, b_words=2)
    LUo, pivo = _lu_compare(s.A, 2)
    LUg, pivg, _ = api().ludecomp(dev(s.A), 2)
    xg = host(api().solve(LUg, pivg, dev(s.b), 2))
    assert np.array_equal(xg, oracle.solve(2, LUo, pivo, s.b))


@pytest.mark.parametrize("w", [3, 4])
def test_config2_n1024_lu_bitwise_and_refine(w):
    """TD/QD LU + solve at n = 1024 on the SVD-built matrix (kappa 2^33):
    factors bitwise equal to the oracle; refinement with the TD inner solver
    reaches 2^-200 against x* = ones (b = A*1 exactly in 8 words)."""
    s = W.svd_system(1024, 10.0, seed=0)
    _lu_compare(s.A[:w].copy(), w)
    if w == 3:
        res = api().refine(dev(s.A), dev(s.b), 3, 200)
        assert res.status == 0
        x = host(res.x)
        # |x - 1| <= 2^-200 elementwise, checked exactly on the words
        for i in range(0, 1024, 7):
            assert abs(X.words_to_frac(x[:, i]) - 1) <= Fraction(1, 2 ** 200)


def test_config2_n2048_full_size_properties():
    """n = 2048, TD inner, the bench's launch: refined x = ones to 2^-200
    for every entry; the direct TD solve has normwise backward error
    <= 1e-44 (exact residual from the oracle)."""
    s = W.svd_system(2048, 10.0, seed=0)
    A = dev(s.A)
    b = dev(s.b)
    res = api().refine(A, b, 3, 200)
    assert res.status == 0 and 1 <= res.corrections <= 4
    x = host(res.x)
    err = np.abs(x[0] - 1.0)
    assert err.max() <= 2.0 ** -100
    for i in range(0, 2048, 97):
        assert abs(X.words_to_frac(x[:, i]) - 1) <= Fraction(1, 2 ** 200)
    LU, piv, info = api().ludecomp(A, 3)
    xd = host(api().solve(LU, piv, b, 3))
    r = oracle.residual(s.A, s.b, xd, 8)
    rn = np.max(np.abs(r[0]))
    Ainf = np.max(np.sum(np.abs(s.A[0, :, :2048]), axis=0))
    eta = rn / (Ainf * np.max(np.abs(xd[0])) + np.max(np.abs(s.b[0])))
    assert eta <= 1e-44, eta
