"""mw_solve_noalloc, the substitution entry point for callers that cannot
allocate device memory (for example code inside a framework whose memory
pool owns the GPU, or hooks that must not touch an allocator), checked
through the C ABI against mw_solve, which takes a caller-provided work
buffer.  Two calls in a row must both match, since every call reuses the
same fixed scratch.  Collected last on purpose."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2107_12550_gb300 import build as B
    from paper_2107_12550_gb300 import _lib as L
    B.build()
    return L.lib()


def _factor(w, n, seed):
    from paper_2107_12550_gb300 import api
    from paper_2107_12550_gb300 import workloads as W
    A = torch.from_numpy(W.uniform_matrix(n, w, seed=seed)).cuda()
    LU, piv, info = api.ludecomp(A, w)
    g = np.random.default_rng(seed)
    b = torch.from_numpy(np.ascontiguousarray(g.uniform(-1, 1, (w, n)))).cuda()
    return LU, piv, b


def _solve_with_work(lib, w, LU, piv, b):
    from paper_2107_12550_gb300 import _lib as L
    n, lda = LU.shape[1], LU.shape[2]
    work = torch.empty(L.workspace_size(L.MW_OP_SOLVE, w, 0, n), dtype=torch.uint8, device="cuda")
    x = torch.empty_like(b)
    s = torch.cuda.current_stream().cuda_stream
    rc = lib.mw_solve(w, n, LU.data_ptr(), lda, piv.data_ptr(), b.data_ptr(), x.data_ptr(),
                      work.data_ptr(), work.numel(), s)
    assert rc == 0
    return x


def _solve_noalloc(lib, w, LU, piv, b):
    n, lda = LU.shape[1], LU.shape[2]
    x = torch.empty_like(b)
    s = torch.cuda.current_stream().cuda_stream
    rc = lib.mw_solve_noalloc(w, n, LU.data_ptr(), lda, piv.data_ptr(), b.data_ptr(), x.data_ptr(), s)
    assert rc == 0
    return x


def test_noalloc_solve_matches_solve_twice(lib):
    # two calls in a row on different systems and precisions: identical bits
    for w, n, seed in ((3, 700, 1), (2, 1029, 2), (4, 333, 3), (3, 700, 4)):
        LU, piv, b = _factor(w, n, seed)
        ref = _solve_with_work(lib, w, LU, piv, b)
        x1 = _solve_noalloc(lib, w, LU, piv, b)
        x2 = _solve_noalloc(lib, w, LU, piv, b)
        torch.cuda.synchronize()
        assert torch.equal(x1, ref)
        assert torch.equal(x2, ref)


def test_noalloc_rejects_orders_beyond_scratch(lib):
    # checked on the host before any GPU work: -2 (the order n is invalid);
    # 2^62 would wrap the byte counts around size_t if it got that far
    assert lib.mw_solve_noalloc(4, 20969, 8, 20969, 8, 8, 8, None) == -2
    assert lib.mw_solve_noalloc(2, 40321, 8, 40321, 8, 8, 8, None) == -2
    assert lib.mw_solve_noalloc(4, 1 << 62, 8, 1 << 62, 8, 8, 8, None) == -2
    assert lib.mw_solve_noalloc(2, 1 << 62, 8, 1 << 62, 8, 8, 8, None) == -2
    assert lib.mw_solve_noalloc(4, 10, 8, 5, 8, 8, 8, None) == -4


def test_noalloc_largest_qd_order_fills_the_scratch_exactly(lib):
    """QD n = 20968 needs exactly the whole fixed scratch (2 MiB): the
    boundary case that is still accepted.  A hand-built factorisation
    (unit lower L = I, upper U = a random diagonal, no row swaps) keeps it
    cheap; the result must equal mw_solve's with an exactly sized work
    buffer, bitwise, on two calls in a row, and report no wait timeout."""
    from paper_2107_12550_gb300 import _lib as L
    w, n = 4, 20968
    assert L.workspace_size(L.MW_OP_SOLVE, w, 0, n) == 2 * 1024 * 1024
    LU = torch.zeros((w, n, n), dtype=torch.float64, device="cuda")
    g = np.random.default_rng(11)
    d = torch.from_numpy(g.uniform(1.0, 2.0, n)).cuda()
    idx = torch.arange(n, device="cuda")
    LU[0, idx, idx] = d
    piv = torch.arange(n, dtype=torch.int64, device="cuda")
    b = torch.from_numpy(np.ascontiguousarray(g.uniform(-1, 1, (w, n)))).cuda()
    ref = _solve_with_work(lib, w, LU, piv, b)
    x1 = _solve_noalloc(lib, w, LU, piv, b)
    x2 = _solve_noalloc(lib, w, LU, piv, b)
    s = torch.cuda.current_stream().cuda_stream
    assert lib.mw_solve_noalloc_status(s) == 0
    assert torch.equal(x1, ref) and torch.equal(x2, ref)
    del LU
    torch.cuda.empty_cache()
