"""The C-ABI library builds, loads and exports every symbol that
include/mwlu.h declares; host-side argument checks answer without touching a
GPU."""
import ctypes

import pytest

from paper_2107_12550_gb300 import _lib as L
from paper_2107_12550_gb300 import build as B


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def test_exports_every_declared_symbol(lib):
    declared = L.declared_symbols()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), name
    assert set(L.SIGNATURES) >= set(declared)


def test_workspace_sizes(lib):
    for prec in (2, 3, 4):
        for n in (0, 1, 100, 2048):
            lu = L.workspace_size(L.MW_OP_LUDECOMP, prec, 0, n)
            sv = L.workspace_size(L.MW_OP_SOLVE, prec, 0, n)
            rf = L.workspace_size(L.MW_OP_REFINE, prec, 0, n)
            assert lu > 0 and sv > 0
            assert rf >= prec * n * n * 8 + sv
            assert lu % 256 == 0 and sv % 256 == 0 and rf % 256 == 0
    out = ctypes.c_size_t(0)
    assert lib.mw_workspace_size(7, 2, 0, 10, ctypes.byref(out)) == -1
    assert lib.mw_workspace_size(0, 5, 0, 10, ctypes.byref(out)) == -2
    assert lib.mw_workspace_size(0, 2, 9, 10, ctypes.byref(out)) == -3
    assert lib.mw_workspace_size(0, 2, 0, -1, ctypes.byref(out)) == -4


def test_argument_checks_need_no_gpu(lib):
    # every call below is rejected before any CUDA call
    assert lib.mw_ludecomp(5, 0, 4, None, 4, None, None, None, 0, None) == -1
    assert lib.mw_ludecomp(2, 3, 4, None, 4, None, None, None, 0, None) == -2
    assert lib.mw_ludecomp(2, 0, -1, None, 4, None, None, None, 0, None) == -3
    assert lib.mw_ludecomp(2, 0, 4, None, 4, None, None, None, 0, None) == -4
    assert lib.mw_ludecomp(2, 0, 4, 8, 3, 8, 8, 8, 1 << 30, None) == -5
    assert lib.mw_ludecomp(2, 0, 4, 8, 4, 8, 8, 8, 16, None) == -9
    assert lib.mw_ludecomp(3, 1, 4, 8, 4, 8, 8, 8, 1 << 30, None) == L.MW_EUNSUPPORTED
    assert lib.mw_solve(1, 4, 8, 4, 8, 8, 8, 8, 1 << 30, None) == -1
    assert lib.mw_solve(2, 4, 8, 2, 8, 8, 8, 8, 1 << 30, None) == -4
    assert lib.mw_residual(4, 8, 4, 9, 8, 1, 8, 1, 8, 1, None) == -4
    assert lib.mw_residual(4, 8, 4, 1, 8, 1, 8, 1, 8, 0, None) == -10
    stats = (ctypes.c_int64 * 4)()
    assert lib.mw_refine(4, 8, 4, 2, 8, 2, 3, 0, 200, 5, 1, 0.0, 0.0, 8, 2, stats, 8, 1 << 30, None) == -15
    assert lib.mw_refine(4, 8, 4, 2, 8, 2, 3, 0, 200, -1, 1, 0.0, 0.0, 8, 8, stats, 8, 1 << 30, None) == -10
    assert lib.mw_arith(9, 2, 4, 8, 8, 8, None) == -1
    assert lib.mw_strerror(L.MW_ESINGULAR).startswith(b"exactly zero pivot")
    assert lib.mw_version().startswith(b"mwlu")


def test_strassen_workspace_argument_checks():
    """mw_gemm_strassen_workspace_size (host only): sizes that the recursion
    cannot split, the split form's DD-only and 64-multiple block rules, and
    invalid arguments."""
    import ctypes
    from paper_2107_12550_gb300 import build as B
    B.build()
    from paper_2107_12550_gb300 import _lib as L
    lib = L.lib()
    nb = ctypes.c_size_t(0)
    assert lib.mw_gemm_strassen_workspace_size(2, 0, 2, 102, ctypes.byref(nb)) == L.MW_EUNSUPPORTED   # 102 % 4
    assert lib.mw_gemm_strassen_workspace_size(2, 1, 1, 192, ctypes.byref(nb)) == L.MW_EUNSUPPORTED   # 96 % 64
    assert lib.mw_gemm_strassen_workspace_size(3, 1, 1, 256, ctypes.byref(nb)) == L.MW_EUNSUPPORTED   # split: DD only
    assert lib.mw_gemm_strassen_workspace_size(5, 0, 1, 64, ctypes.byref(nb)) == -1
    assert lib.mw_gemm_strassen_workspace_size(2, 2, 1, 64, ctypes.byref(nb)) == -2
    assert lib.mw_gemm_strassen_workspace_size(2, 0, 9, 512, ctypes.byref(nb)) == -3
    assert lib.mw_gemm_strassen_workspace_size(2, 0, 1, 64, None) == -5
    # levels 2 at n = 256, plain DD: 9 x 2 x (128^2 + 64^2) doubles after a 256-byte header
    assert lib.mw_gemm_strassen_workspace_size(2, 0, 2, 256, ctypes.byref(nb)) == 0
    assert nb.value == 256 + 8 * 9 * 2 * (128 * 128 + 64 * 64)


def test_python_binding_rejects_host_and_mismatched_operands():
    """The binding checks device, dtype and shapes before any library call
    (no GPU needed to see the errors)."""
    import torch
    import pytest as _pt
    from paper_2107_12550_gb300 import api
    A = torch.zeros((2, 8, 8), dtype=torch.float64)          # host tensor
    with _pt.raises(ValueError):
        api.gemm_strassen(A, A, 2, "plain", 1)
    with _pt.raises(ValueError):
        api.ludecomp(A, 2)
    with _pt.raises(ValueError):
        api.gemm_sub(A, A, A, 8, 2)


def test_huge_orders_rejected_before_any_size_arithmetic(lib):
    """Orders far beyond any device (here 2^62, whose byte counts would wrap
    around size_t) are rejected on the host as invalid arguments."""
    big = 1 << 62
    out = ctypes.c_size_t(0)
    assert lib.mw_workspace_size(L.MW_OP_SOLVE, 4, 0, big, ctypes.byref(out)) == -4
    assert lib.mw_ludecomp(2, 0, big, 8, big, 8, 8, 8, 1 << 30, None) == -3
    assert lib.mw_solve(4, big, 8, big, 8, 8, 8, 8, 1 << 30, None) == -2
    assert lib.mw_solve_noalloc(4, big, 8, big, 8, 8, 8, None) == -2
    assert lib.mw_solve_noalloc(2, 40321, 8, 40321, 8, 8, 8, None) == -2
    assert lib.mw_residual(big, 8, big, 1, 8, 1, 8, 1, 8, 1, None) == -1
    stats = (ctypes.c_int64 * 4)()
    assert lib.mw_refine(big, 8, big, 2, 8, 2, 3, 0, 200, 5, 1, 0.0, 0.0, 8, 8, stats, 8, 1 << 30, None) == -1
    assert lib.mw_gemm_sub(2, 0, big, 4, 4, 8, big, 8, big, 8, 4, None, 0, None) == -3
    # element counts whose grid would not fit the launch's x extent
    assert lib.mw_arith(0, 2, big, 8, 8, 8, None) == -3
    assert lib.mw_arith(0, 2, 256 * (2**31 - 1) + 1, 8, 8, 8, None) == -3
    assert lib.mw_arith(0, 2, 2**63 - 1, 8, 8, 8, None) == -3


def test_order_bound_keeps_every_size_exact(lib):
    """Orders and leading dimensions are bounded by 2^28: just above it every
    entry point rejects the call on the host; at it, the byte counts that
    grow with n^2 (the refinement's LU copy, Strassen's temporaries) are
    still exact, not wrapped around size_t."""
    top = 1 << 28
    out = ctypes.c_size_t(0)
    assert lib.mw_workspace_size(L.MW_OP_REFINE, 4, 0, top + 1, ctypes.byref(out)) == -4
    assert lib.mw_workspace_size(L.MW_OP_REFINE, 4, 0, top, ctypes.byref(out)) == 0
    assert out.value >= 8 * 4 * top * top                  # the QD LU copy alone
    for bad in (top + 2, 1 << 62):
        assert lib.mw_gemm_strassen_workspace_size(4, 0, 1, bad, ctypes.byref(out)) == -4
        assert lib.mw_gemm_strassen(4, 0, 1, bad, 8, bad, 8, bad, 8, bad, 8, 1 << 30, None) == -4
    assert lib.mw_gemm_strassen_workspace_size(4, 0, 1, top, ctypes.byref(out)) == 0
    assert out.value >= 8 * 9 * 4 * (top // 2) ** 2        # one level of temporaries
    # leading dimensions above the bound, with small orders
    ld = top + 1
    stats = (ctypes.c_int64 * 4)()
    assert lib.mw_ludecomp(2, 0, 8, 8, ld, 8, 8, 8, 1 << 30, None) == -5
    assert lib.mw_solve(2, 8, 8, ld, 8, 8, 8, 8, 1 << 30, None) == -4
    assert lib.mw_solve_noalloc(2, 8, 8, ld, 8, 8, 8, None) == -4
    assert lib.mw_residual(8, 8, ld, 1, 8, 1, 8, 1, 8, 1, None) == -3
    assert lib.mw_refine(8, 8, ld, 2, 8, 2, 3, 0, 200, 5, 1, 0.0, 0.0, 8, 8, stats, 8, 1 << 30, None) == -3
    assert lib.mw_gemm_sub(2, 0, 8, 8, 8, 8, ld, 8, 8, 8, 8, None, 0, None) == -7
    assert lib.mw_gemm_sub(2, 0, 8, 8, 8, 8, 8, 8, ld, 8, 8, None, 0, None) == -9
    assert lib.mw_gemm_sub(2, 0, 8, 8, 8, 8, 8, 8, 8, 8, ld, None, 0, None) == -11
    assert lib.mw_gemm_strassen(2, 0, 1, 64, 8, ld, 8, 64, 8, 64, 8, 1 << 30, None) == -6
    assert lib.mw_gemm_strassen(2, 0, 1, 64, 8, 64, 8, 64, 8, ld, 8, 1 << 30, None) == -10


def test_batched_arguments_checked_on_the_host(lib):
    """The batched entry points check their arguments, orders included
    (1 <= n <= 1024), before any device work; an empty batch is a no-op."""
    def orders(*ns):
        return (ctypes.c_int * len(ns))(*ns)
    out = ctypes.c_size_t(0)
    ok2, bad_hi, bad_lo = orders(3, 5), orders(3, 1025), orders(0, 5)
    # sizes
    assert lib.mw_batch_workspace_size(L.MW_OP_SOLVE, 2, 2, ok2, ctypes.byref(out)) == 0 and out.value > 0
    assert lib.mw_batch_workspace_size(9, 2, 2, ok2, ctypes.byref(out)) == -1
    assert lib.mw_batch_workspace_size(L.MW_OP_SOLVE, 5, 2, ok2, ctypes.byref(out)) == -2
    assert lib.mw_batch_workspace_size(L.MW_OP_SOLVE, 2, -1, ok2, ctypes.byref(out)) == -3
    assert lib.mw_batch_workspace_size(L.MW_OP_SOLVE, 2, 2, bad_hi, ctypes.byref(out)) == -4
    assert lib.mw_batch_workspace_size(L.MW_OP_SOLVE, 2, 2, bad_lo, ctypes.byref(out)) == -4
    assert lib.mw_batch_workspace_size(L.MW_OP_SOLVE, 2, 2, ok2, None) == -5
    assert lib.mw_batch_blocked_workspace_size(L.MW_OP_REFINE, 2, 1, 2, ok2, ctypes.byref(out)) == 0
    assert lib.mw_batch_blocked_workspace_size(L.MW_OP_LUDECOMP, 3, 1, 2, ok2, ctypes.byref(out)) \
        == L.MW_EUNSUPPORTED                                   # split update is DD only
    assert lib.mw_batch_blocked_workspace_size(L.MW_OP_LUDECOMP, 2, 0, 2, bad_hi, ctypes.byref(out)) == -5
    # factorisation, substitution, refinement
    big = 1 << 30
    assert lib.mw_ludecomp_batched(2, 0, None, None, None, None, None, 0, None) == 0
    assert lib.mw_ludecomp_batched(2, 2, bad_hi, 8, 8, 8, 8, big, None) == -3
    assert lib.mw_ludecomp_batched_blocked(2, 0, 2, bad_lo, 8, 8, 8, 8, big, None) == -4
    assert lib.mw_ludecomp_batched_blocked(3, 1, 2, ok2, 8, 8, 8, 8, big, None) == L.MW_EUNSUPPORTED
    assert lib.mw_ludecomp_batched_blocked(2, 0, 2, ok2, 8, 8, 8, 8, 0, None) == -9
    assert lib.mw_solve_batched(2, 2, bad_lo, 8, 8, 8, 8, 8, big, None) == -3
    assert lib.mw_solve_batched(2, 2, ok2, 8, 8, 8, 8, 8, 0, None) == -9
    assert lib.mw_refine_batched(2, ok2, 8, 9, 8, 8, 2, 200, 30, 8, 8, 8, 8, big, None) == -4
    assert lib.mw_refine_batched(2, ok2, 8, 4, 8, 8, 3, 200, 30, 8, 2, 8, 8, big, None) == -11
    assert lib.mw_refine_batched(2, bad_hi, 8, 4, 8, 8, 2, 200, 30, 8, 8, 8, 8, big, None) == -2
    assert lib.mw_refine_batched(2, ok2, 8, 4, 8, 8, 2, 200, 30, 8, 8, 8, 8, 0, None) == -14
    assert lib.mw_refine_batched_blocked(2, ok2, 8, 4, 8, 8, 3, 1, 200, 30, 8, 8, 8, 8, big, None) \
        == L.MW_EUNSUPPORTED
    assert lib.mw_refine_batched_blocked(2, bad_hi, 8, 4, 8, 8, 2, 1, 200, 30, 8, 8, 8, 8, big, None) == -2
    assert lib.mw_refine_batched_blocked(2, ok2, 8, 4, 8, 8, 2, 1, 0, 30, 8, 8, 8, 8, big, None) == -9
    assert lib.mw_refine_batched_blocked(2, ok2, 8, 4, 8, 8, 2, 1, 200, 30, 8, 8, 8, 8, 0, None) == -15


def test_status_and_wait_limit_arguments(lib):
    assert lib.mw_work_status(7, 0, 8, None) == -1
    assert lib.mw_work_status(L.MW_OP_SOLVE, 5, 8, None) == -2
    assert lib.mw_work_status(L.MW_OP_SOLVE, 0, None, None) == -3
    assert lib.mw_batch_work_status(None, None) == -1
    assert lib.mw_set_wait_limit(-1) == -1
    prev = lib.mw_set_wait_limit(1000)
    assert prev == 0
    assert lib.mw_set_wait_limit(prev) == 1000


def test_build_compiles_every_translation_unit():
    """Every .cu file of the library is in the build's source list (a file
    left out would leave its kernels' symbols undefined only at load time)."""
    import os
    from paper_2107_12550_gb300 import build as B
    on_disk = sorted(f for f in os.listdir(B.CSRC) if f.endswith(".cu"))
    assert sorted(B.SOURCES) == on_disk
