"""Bounded device waits and their error reporting, through the C ABI.

With the poll limit lowered by mw_set_wait_limit, real waits run out: the
substitution's polls for other warps' published rows, the panel's waits
for every CTA's candidate record, the batched substitution's waits between
its leader and worker warps.  Each kernel then records the error word and
returns (nothing faults or hangs: every wait is bounded, and the kernels
only leave their outputs incomplete).  The status calls report MW_ETIMEOUT,
and the next call with the default limit is bitwise equal to the result
before (which the parity tests pin to the oracle)."""
import numpy as np
import pytest

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


@pytest.fixture
def short_waits():
    """Lowers the poll limit to 1 for the test body, restores it after."""
    def lower():
        return api().set_wait_limit(1)
    prev = api().set_wait_limit(0)
    yield lower
    api().set_wait_limit(prev)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_solve_wait_runs_out_then_recovers(short_waits):
    n, w = 1024, 3
    A = dev(W.uniform_matrix(n, w, seed=3))
    LU, piv, info = api().ludecomp(A, w)
    b = dev(np.random.default_rng(3).uniform(-1, 1, (w, n)))
    work = api().workspace(L.MW_OP_SOLVE, w, 0, n)
    ref = api().solve(LU, piv, b, w, work=work).clone()
    assert api().work_status(L.MW_OP_SOLVE, "plain", work) == L.MW_OK
    short_waits()
    api().solve(LU, piv, b, w, work=work)
    assert api().work_status(L.MW_OP_SOLVE, "plain", work) == L.MW_ETIMEOUT
    api().set_wait_limit(0)
    x = api().solve(LU, piv, b, w, work=work)
    assert api().work_status(L.MW_OP_SOLVE, "plain", work) == L.MW_OK
    assert torch.equal(x, ref)


def test_panel_wait_runs_out_then_recovers(short_waits):
    n, w = 1024, 2
    A = dev(W.uniform_matrix(n, w, seed=4))
    work = api().workspace(L.MW_OP_LUDECOMP, w, 0, n)
    LU0, piv0, _ = api().ludecomp(A, w, work=work)
    LU0, piv0 = LU0.clone(), piv0.clone()
    short_waits()
    api().ludecomp(A, w, work=work)
    assert api().work_status(L.MW_OP_LUDECOMP, "plain", work) == L.MW_ETIMEOUT
    api().set_wait_limit(0)
    LU1, piv1, info = api().ludecomp(A, w, work=work)
    assert api().work_status(L.MW_OP_LUDECOMP, "plain", work) == L.MW_OK
    assert torch.equal(LU1, LU0) and torch.equal(piv1, piv0) and int(info.item()) == 0


def test_refine_returns_timeout(short_waits):
    s = W.svd_system(512, 8.0, seed=5)
    A, b = dev(s.A), dev(s.b)
    ok = api().refine(A, b, 3, 200)
    assert ok.status == L.MW_OK
    short_waits()
    with pytest.raises(L.MWError) as e:
        api().refine(A, b, 3, 200)
    assert e.value.code == L.MW_ETIMEOUT
    api().set_wait_limit(0)
    again = api().refine(A, b, 3, 200)
    assert again.status == L.MW_OK and torch.equal(again.x, ok.x)


def test_batched_solve_wait_runs_out_then_recovers(short_waits):
    n_list = [700, 300, 512, 64]
    mats = [W.uniform_matrix(m, 2, seed=W.system_seed(9, s), lda=m) for s, m in enumerate(n_list)]
    vecs = [np.random.default_rng(s).uniform(-1, 1, (2, m)) for s, m in enumerate(n_list)]
    A = dev(api().pack_matrices(mats, 2))
    b = dev(api().pack_vectors(vecs, 2))
    work = api().batch_workspace(L.MW_OP_LUDECOMP, 2, n_list)
    LU, piv, info = api().ludecomp_batched(A, n_list, 2, work=work)
    ref = api().solve_batched(LU, piv, b, n_list, 2, work=work).clone()
    assert api().batch_work_status(work) == L.MW_OK
    short_waits()
    api().solve_batched(LU, piv, b, n_list, 2, work=work)
    assert api().batch_work_status(work) == L.MW_ETIMEOUT
    api().set_wait_limit(0)
    x = api().solve_batched(LU, piv, b, n_list, 2, work=work)
    assert api().batch_work_status(work) == L.MW_OK
    assert torch.equal(x, ref)
