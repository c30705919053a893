"""The seeded input generators: shapes, exactness of b = A x_true, canonical
words, and the condition number of the SVD-built matrices (Section 3,
Eq. (1) and the synthetic stand-ins for it)."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import exact as X
from paper_2107_12550_gb300 import workloads as W


def test_uniform_words_canonical_and_seeded():
    A = W.uniform_matrix(40, 3, seed=1)
    B = W.uniform_matrix(40, 3, seed=1)
    assert np.array_equal(A, B)
    assert A.shape == (3, 40, 64)
    assert np.all(A[:, :, 40:] == 0)
    for c in range(2):
        hi, lo = A[c, :, :40].ravel(), A[c + 1, :, :40].ravel()
        assert np.all(hi + lo == hi)          # canonical: RN(hi + lo) = hi
    assert np.abs(A[0]).max() <= 1.0


def test_rowsum_greedy_exact():
    A = W.uniform_matrix(9, 2, seed=2, lda=9)
    b = W.rowsum_words(A, None, 3)
    Af = X.mat_to_frac(A, 9)
    for i in range(9):
        assert list(b[:, i]) == X.greedy_words(sum(Af[i]), 3)


def test_svd_system_exact_b_and_condition():
    s = W.svd_system(30, 6.0, seed=4)
    Af = X.mat_to_frac(s.A, 30)
    bf = X.vec_to_frac(s.b)
    assert all(sum(row) == bi for row, bi in zip(Af, bf))    # b = A * ones exactly
    for i in range(30):
        for j in range(30):
            assert list(s.A[:, j, i]) == X.greedy_words(Af[i][j], 4)
    sv = np.linalg.svd(s.A[0, :, :30].T, compute_uv=False)
    E = round(math.log2(10) * 6.0)
    assert abs(math.log2(sv[0] / sv[-1]) - E) < 0.01


def test_paper_system_exact_b():
    s = W.paper_system(20, seed=1)
    Af = X.mat_to_frac(s.A, 20)
    xs = [Fraction(int(v)) for v in s.x_star]
    assert X.matvec(Af, xs) == X.vec_to_frac(s.b)
    assert list(s.x_star) == list(range(20))


def test_batch_sizes_range():
    n = W.batch_sizes(1000, 16, 256, seed=0)
    assert n.min() >= 16 and n.max() <= 256
    assert np.array_equal(n, W.batch_sizes(1000, 16, 256, seed=0))


def test_mixed_batch_spec_ranges():
    n_list, kap = W.mixed_batch_spec(512, 64, 1024, 4.0, 20.0, seed=0)
    assert len(n_list) == len(kap) == 512
    assert min(n_list) >= 64 and max(n_list) <= 1024
    assert min(kap) >= 4.0 and max(kap) <= 20.0
    assert (n_list, kap) == W.mixed_batch_spec(512, 64, 1024, 4.0, 20.0, seed=0)


@pytest.mark.timeout(300)
def test_svd_batch_pool_matches_single_systems():
    """The packed batch built by worker processes equals the one built in
    this process and, system by system, svd_system with its per-system seed;
    b = A * ones exactly for a sampled small member."""
    n_list, kap = W.mixed_batch_spec(10, 5, 40, 4.0, 20.0, seed=9)
    A, b = W.svd_batch(n_list, kap, seed=9, processes=2)
    A1, b1 = W.svd_batch(n_list, kap, seed=9, processes=1)
    assert np.array_equal(A, A1) and np.array_equal(b, b1)
    n = np.asarray(n_list)
    moff = np.concatenate([[0], np.cumsum(n * n)])
    voff = np.concatenate([[0], np.cumsum(n)])
    for s, ns in enumerate(n_list):
        ref = W.svd_system(ns, kap[s], seed=W.system_seed(9, s), lda=ns)
        assert np.array_equal(A[4 * moff[s]: 4 * moff[s + 1]].reshape(4, ns, ns), ref.A)
        assert np.array_equal(b[8 * voff[s]: 8 * voff[s + 1]].reshape(8, ns), ref.b)
    s = int(np.argmin(n))
    Af = X.mat_to_frac(A[4 * moff[s]: 4 * moff[s + 1]].reshape(4, n[s], n[s]), int(n[s]))
    bf = X.vec_to_frac(b[8 * voff[s]: 8 * voff[s + 1]].reshape(8, n[s]))
    assert all(sum(row) == bi for row, bi in zip(Af, bf))
