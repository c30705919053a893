"""The Python binding hands every tensor to the library as a raw device
address with no extent attached, so it checks each one first: a host tensor,
another GPU's, the wrong element type, too few planes or elements raise
ValueError before any allocation or library call.  Valid calls, shaped like
those of the GPU tests, pass the checks and reach the library.

Runs without a GPU: device tensors are stood in for by objects carrying
only what the checks read (shape, element type, device, contiguity)."""
import math
from types import SimpleNamespace

import pytest
import torch

from paper_2107_12550_gb300 import _lib as L
from paper_2107_12550_gb300 import api


class Dev:
    """Stand-in for a CUDA tensor."""
    is_cuda = True

    def __init__(self, *shape, dtype=torch.float64, device="cuda:0", contiguous=True, ptr=None):
        self.shape = torch.Size(shape)
        self.dtype = dtype
        self.device = torch.device(device)
        self._contiguous = contiguous
        self._ptr = ptr

    def dim(self):
        return len(self.shape)

    def numel(self):
        return math.prod(self.shape)

    def is_contiguous(self):
        return self._contiguous

    def element_size(self):
        return torch.empty(0, dtype=self.dtype).element_size()

    def data_ptr(self):
        if self._ptr is None:
            raise AssertionError("a device address was taken on a call that should have been rejected")
        return self._ptr


def I64(*shape, **kw):
    return Dev(*shape, dtype=torch.int64, **kw)


def WORK(count=1 << 20, dtype=torch.uint8, **kw):
    return Dev(count, dtype=dtype, **kw)


STREAM = SimpleNamespace(cuda_stream=0)


@pytest.fixture
def no_library(monkeypatch):
    def fail():
        raise AssertionError("the library was called")
    monkeypatch.setattr(L, "lib", fail)


@pytest.fixture
def recorder(monkeypatch):
    calls = []

    class Lib:
        def __getattr__(self, name):
            def fn(*args):
                calls.append((name, args))
                return 0
            return fn
    monkeypatch.setattr(L, "lib", lambda: Lib())
    return calls


def with_ptrs(*ts):
    for k, t in enumerate(ts):
        t._ptr = 4096 * (k + 1)
    return ts


n, w, lda = 8, 2, 11


@pytest.mark.parametrize("case", [
    # host tensors where device addresses are taken
    lambda: api.solve(Dev(w, n, lda), torch.zeros(n, dtype=torch.int64), Dev(w, n), w),
    lambda: api.solve(Dev(w, n, lda), I64(n), Dev(w, n), w, work=torch.empty(64, dtype=torch.uint8)),
    lambda: api.ludecomp(Dev(w, n, lda), w, work=torch.empty(64, dtype=torch.uint8)),
    # wrong element type, too few pivots, too few planes
    lambda: api.solve(Dev(w, n, lda), Dev(n, dtype=torch.int32), Dev(w, n), w),
    lambda: api.solve(Dev(w, n, lda), I64(n - 1), Dev(w, n), w),
    lambda: api.solve(Dev(w, n, lda), I64(n), Dev(w, n), 3),
    # right-hand side or output of the wrong extent, another device
    lambda: api.solve(Dev(w, n, lda), I64(n), Dev(w, n + 1), w),
    lambda: api.solve(Dev(w, n, lda), I64(n), Dev(w, n, device="cuda:1"), w),
    lambda: api.solve(Dev(w, n, lda), I64(n), Dev(w, n), w, out=Dev(w, n - 1)),
    lambda: api.solve(Dev(w, n, lda), I64(n, device="cuda:1"), Dev(w, n), w),
    lambda: api.solve(Dev(w, n, lda), I64(n), Dev(w, n), w, work=WORK(device="cuda:1")),
    lambda: api.residual(Dev(4, n, lda), Dev(1, n), Dev(3, n + 1), 8),
    lambda: api.residual(Dev(4, n, lda), Dev(1, n), Dev(3, n), 8, out=Dev(8 * n - 1)),
    lambda: api.refine(Dev(4, n, lda), Dev(8, n - 1), 3),
    lambda: api.refine(Dev(4, n, lda), Dev(8, n), 3, out=Dev(7, n)),
    lambda: api.refine(Dev(4, n, lda), Dev(8, n), 3, work=WORK(contiguous=False)),
    # block products: B's columns, planes, devices
    lambda: api.gemm_sub(Dev(2, 40, 153), Dev(2, 128, 153), Dev(2, 41, 131), 150, 2),
    lambda: api.gemm_sub(Dev(2, 40, 153), Dev(1, 128, 153), Dev(2, 40, 131), 150, 2),
    lambda: api.gemm_add(Dev(2, 40, 153), Dev(2, 128, 153, device="cuda:1"), Dev(2, 40, 131), 150, 2),
    lambda: api.gemm(Dev(2, 128, 153), Dev(1, 40, 131), 150, 2),
    lambda: api.gemm_strassen(Dev(2, 64, 64), Dev(2, 64, 64, device="cuda:1"), 2),
    # batches: n = 3 and 5, so sum n = 8 and sum n^2 = 34
    lambda: api.ludecomp_batched(Dev(2 * 34 - 1), [3, 5], 2),
    lambda: api.ludecomp_batched(torch.zeros(2 * 34, dtype=torch.float64), [3, 5], 2),
    lambda: api.ludecomp_batched_blocked(Dev(2 * 34, dtype=torch.float32), [3, 5], 2, "split"),
    lambda: api.solve_batched(Dev(2 * 34), I64(7), Dev(2 * 8), [3, 5], 2),
    lambda: api.solve_batched(Dev(2 * 34), I64(8), Dev(2 * 8 - 1), [3, 5], 2),
    lambda: api.solve_batched(Dev(2 * 34), I64(8), Dev(2 * 8), [3, 5], 2, out=Dev(15)),
    lambda: api.solve_batched(Dev(3 * 34 - 1), I64(8), Dev(3 * 8), [3, 5], 3),
    lambda: api.refine_batched(Dev(4 * 34 - 1), 4, Dev(8 * 8), 8, [3, 5], 2),
    lambda: api.refine_batched_blocked(Dev(4 * 34), 4, Dev(8 * 8 - 1), 8, [3, 5], 2, "split"),
    lambda: api.refine_batched_blocked(Dev(4 * 34), 4, Dev(8 * 8), 8, [3, 5], 2, "split", out=Dev(8 * 8 - 1)),
    lambda: api.refine_batched_blocked(Dev(4 * 34), 0, Dev(8 * 8), 8, [3, 5], 2, "split"),
    lambda: api.refine_batched_blocked(Dev(4 * 34), 4, Dev(8 * 8, device="cuda:1"), 8, [3, 5], 2),
    # element-wise operands and status queries
    lambda: api.arith(0, 2, Dev(2, 100), Dev(2, 99)),
    lambda: api.arith(0, 3, Dev(2, 100), Dev(2, 100)),
    lambda: api.work_status(L.MW_OP_SOLVE, "plain", torch.empty(256, dtype=torch.uint8)),
    lambda: api.batch_work_status(torch.empty(256, dtype=torch.uint8)),
])
def test_rejected_before_the_library(no_library, case):
    with pytest.raises(ValueError):
        case()


def test_valid_single_system_calls_reach_the_library(recorder):
    LU, piv, b, x, work = with_ptrs(Dev(w, n, lda), I64(n), Dev(w, n), Dev(w, n), WORK(4096, dtype=torch.float64))
    assert api.solve(LU, piv, b, w, out=x, work=work, stream=STREAM) is x
    name, args = recorder[-1]
    assert name == "mw_solve" and args[:2] == (w, n) and args[3] == lda
    assert args[-2] == 4096 * 8                      # bytes, whatever the work buffer's element type
    # x aliased with b (the substitution runs in place)
    assert api.solve(LU, piv, b, w, out=b, work=work, stream=STREAM) is b
    A, bb, xx, r = with_ptrs(Dev(4, n, lda), Dev(1, n), Dev(3, n), Dev(8, n))
    assert api.residual(A, bb, xx, 8, out=r, stream=STREAM) is r
    assert recorder[-1][1][:4] == (n, A._ptr, lda, 4)
    A, b8, x8, work = with_ptrs(Dev(4, n, lda), Dev(8, n), Dev(8, n), WORK())
    res = api.refine(A, b8, 3, 200, out=x8, work=work, stream=STREAM)
    assert res.x is x8 and recorder[-1][0] == "mw_refine"
    C, A, B, work = with_ptrs(Dev(2, 40, 153), Dev(2, 128, 153), Dev(2, 40, 131), WORK())
    assert api.gemm_sub(C, A, B, 150, 2, work=work, stream=STREAM) is C
    assert recorder[-1][1][:5] == (2, 0, 150, 40, 128)


def test_valid_batched_solve_reaches_the_library(recorder):
    LU, piv, b, x, work = with_ptrs(Dev(2 * 34), I64(8), Dev(2 * 8), Dev(2 * 8), WORK())
    assert api.solve_batched(LU, piv, b, [3, 5], 2, out=x, work=work, stream=STREAM) is x
    name, args = recorder[-1]
    assert name == "mw_solve_batched" and args[0] == 2 and args[1] == 2
