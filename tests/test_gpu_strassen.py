"""Strassen's recursion over the block matrix product on the GPU
(mw_gemm_strassen) against the oracle's recursion (oracle/strassen.py):
bitwise for the plain form, within the Strassen error bound of the exact
product for the split form."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import exact as X
from oracle import strassen as S

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2107_12550_gb300 import build as B
    B.build()


def api():
    from paper_2107_12550_gb300 import api as A
    return A


def _mw_mat(w, n, seed, ld=None):
    g = np.random.default_rng(seed)
    ld = ld or n
    M = np.zeros((w, n, ld))
    M[0, :, :n] = g.uniform(-1, 1, (n, n))
    for c in range(1, w):
        _, ex = np.frexp(M[c - 1, :, :n])
        M[c, :, :n] = np.ldexp(g.uniform(-1, 1, (n, n)), ex - 54)
    return M


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n,levels", [(128, 0), (128, 1), (128, 2), (96, 1), (64, 3)])
@pytest.mark.parametrize("w", [2, 3, 4])
def test_plain_bitwise_against_oracle(w, n, levels):
    A = _mw_mat(w, n, 100 + n + levels)
    B = _mw_mat(w, n, 200 + n + levels)
    got = api().gemm_strassen(_dev(A), _dev(B), w, "plain", levels)
    torch.cuda.synchronize()
    ref = S.strassen(w, A, B, levels)
    assert np.array_equal(got.cpu().numpy()[:, :, :n], ref)


def test_plain_strided_operands():
    """Leading dimensions larger than n on every operand."""
    w, n, levels = 3, 64, 2
    A = _mw_mat(w, n, 7, ld=70)
    B = _mw_mat(w, n, 8, ld=67)
    out = torch.zeros((w, n, 75), dtype=torch.float64, device="cuda")
    api().gemm_strassen(_dev(A), _dev(B), w, "plain", levels, out=out)
    torch.cuda.synchronize()
    ref = S.strassen(w, np.ascontiguousarray(A[:, :, :n]), np.ascontiguousarray(B[:, :, :n]), levels)
    assert np.array_equal(out.cpu().numpy()[:, :, :n], ref)


@pytest.mark.parametrize("levels", [1, 2])
def test_split_within_strassen_bound(levels):
    """Split DD base products: the error against the exact product stays
    within Higham's Strassen bound with u = 2^-100 (sampled entries)."""
    n = 256
    A = _mw_mat(2, n, 300 + levels)
    B = _mw_mat(2, n, 400 + levels)
    got = api().gemm_strassen(_dev(A), _dev(B), 2, "split", levels).cpu().numpy()
    n0 = n >> levels
    growth = (n / n0) ** np.log2(12) * (n0 ** 2 + 5 * n0) - 5 * n
    amax, bmax = np.max(np.abs(A[0])), np.max(np.abs(B[0]))
    bound = Fraction(growth) * Fraction(2) ** -100 * Fraction(amax) * Fraction(bmax)
    for i in range(0, n, 37):
        for j in range(0, n, 41):
            xs = np.concatenate([A[0, :, i], A[0, :, i], A[1, :, i], A[1, :, i]])
            ys = np.concatenate([B[0, j, :], B[1, j, :], B[0, j, :], B[1, j, :]])
            exact = X.words_to_frac(oracle.exact_dot(xs, ys, 4))
            assert abs(X.words_to_frac(got[:, j, i]) - exact) <= bound
