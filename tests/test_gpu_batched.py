"""Batched form: many independent systems of uneven order in one launch per
step, through the C ABI.  Each system's factors, pivots, solutions and
refined solutions must be bitwise identical to the CPU oracle's
single-system results (sampled systems at the full batch sizes)."""

import numpy as np
import pytest

import oracle
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


def _uniform_batch(w, n_list, seed):
    mats = [W.uniform_matrix(int(n), w, seed=W.system_seed(seed, s), lda=int(n)) for s, n in enumerate(n_list)]
    vecs = [W.uniform_matrix(int(n), 1, seed=W.system_seed(seed + 1, s), lda=int(n))[0, :1, :] for s, n in
            enumerate(n_list)]
    vecs = [np.vstack([v, np.zeros((w - 1, v.shape[1]))]) for v in vecs]
    return mats, vecs


@pytest.mark.parametrize("w", [2, 3, 4])
def test_lu_and_solve_batched_bitwise(w):
    n_list = [int(v) for v in W.batch_sizes(40, 1, 70, seed=w)]
    n_list[:3] = [1, 2, 33]
    mats, vecs = _uniform_batch(w, n_list, seed=10 * w)
    A = dev(api().pack_matrices(mats, w))
    b = dev(api().pack_vectors(vecs, w))
    LU, piv, info = api().ludecomp_batched(A, n_list, w)
    x = api().solve_batched(LU, piv, b, n_list, w)
    LUs = api().unpack_matrices(host(LU), n_list, w)
    xs = api().unpack_vectors(host(x), n_list, w)
    _, voff = api().batch_offsets(n_list)
    pv = host(piv)
    inf = host(info)
    for s, n in enumerate(n_list):
        LUo, pivo, infoo = oracle.lu(w, mats[s])
        assert np.array_equal(LUs[s], LUo[:, :, :n].transpose(0, 1, 2)), s
        assert np.array_equal(pv[voff[s]: voff[s] + n], pivo), s
        assert inf[s] == infoo
        assert np.array_equal(xs[s], oracle.solve(w, LUo, pivo, vecs[s])), s


def test_batched_singular_member():
    w = 2
    n_list = [20, 7, 31]
    mats, vecs = _uniform_batch(w, n_list, seed=3)
    mats[1][:, 4, :] = 0.0          # zero column: a zero pivot at step 5 at the latest
    A = dev(api().pack_matrices(mats, w))
    LU, piv, info = api().ludecomp_batched(A, n_list, w)
    inf = host(info)
    for s in range(3):
        assert inf[s] == oracle.lu(w, mats[s])[2]
    assert inf[1] > 0 and inf[0] == 0 and inf[2] == 0


@pytest.mark.parametrize("inner", [2, 3])
def test_refine_batched_bitwise(inner):
    n_list = [24, 5, 61, 33, 1, 47]
    systems = [W.svd_system(n, [4.0, 8.0, 12.0][s % 3], seed=100 + s) if n > 1 else
               W.System(np.array([[[3.0]]]), np.array([[1.0]] + [[0.0]] * 7), None) for s, n in enumerate(n_list)]
    A = dev(api().pack_matrices([s.A for s in systems], 4))
    b = dev(api().pack_vectors([s.b for s in systems], 8))
    x, stats = api().refine_batched(A, 4, b, 8, n_list, inner, 200)
    xs = api().unpack_vectors(host(x), n_list, 8)
    st = host(stats)
    for s, sysm in enumerate(systems):
        status, xo, corr, nres, info = oracle.refine(sysm.A, sysm.b, inner)
        assert (st[s, 0], st[s, 1], st[s, 2], st[s, 3]) == (corr, nres, info, status), s
        assert np.array_equal(xs[s], xo), s


@pytest.mark.parametrize("w", [2, 3])
def test_config4_batch_4096_sampled(w):
    """4096 DD and TD systems, n uniform in [16, 256] (uniform entries, one
    RHS from x_true = ones), the bench's launch: one batched LU + solve; 12
    sampled systems (including the largest and smallest) are bitwise equal
    to the oracle."""
    n_list = [int(v) for v in W.batch_sizes(4096, 16, 256, seed=0)]
    mats, vecs = [], []
    for s, n in enumerate(n_list):
        mats.append(W.uniform_matrix(n, w, seed=W.system_seed(0, s), lda=n))
    for s, n in enumerate(n_list):
        v = np.zeros((w, n))
        v[0] = 1.0
        vecs.append(v)
    A = dev(api().pack_matrices(mats, w))
    b = dev(api().pack_vectors(vecs, w))
    LU, piv, info = api().ludecomp_batched(A, n_list, w)
    x = api().solve_batched(LU, piv, b, n_list, w)
    LUs = api().unpack_matrices(host(LU), n_list, w)
    xs = api().unpack_vectors(host(x), n_list, w)
    order = np.argsort(n_list)
    sample = list(order[:4]) + list(order[-4:]) + [0, 1, 2, 3]
    for s in sample:
        LUo, pivo, infoo = oracle.lu(w, mats[s])
        assert np.array_equal(LUs[s], LUo[:, :, :n_list[s]]), s
        assert np.array_equal(xs[s], oracle.solve(w, LUo, pivo, vecs[s])), s
    assert int(host(info).max()) == 0
