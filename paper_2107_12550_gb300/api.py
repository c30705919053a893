"""Python binding of the C ABI with the paper's call names: ``ludecomp``,
``solve``, ``residual`` and ``refine`` (Section 2, Listing 1).

Argument marshalling only: every step runs in the CUDA library.  Tensors are
torch float64 CUDA tensors in the component-planar layout of
``include/mwlu.h``: a matrix is (w, n, lda) with ``A[c, j, i]`` = word c of
A(i, j), a vector is (w, n).  Work buffers are allocated here with torch and
passed down; the library itself never allocates.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Optional

import torch

from . import _lib as L

PREC = {"dd": L.MW_DD, "td": L.MW_TD, "qd": L.MW_QD, 2: L.MW_DD, 3: L.MW_TD, 4: L.MW_QD}
UPDATE = {"plain": L.MW_UPDATE_PLAIN, "split": L.MW_UPDATE_SPLIT, 0: 0, 1: 1}


def _prec(p) -> int:
    return PREC[p.lower() if isinstance(p, str) else p]


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _check_mat(A: torch.Tensor, name: str):
    if not (A.is_cuda and A.dtype == torch.float64 and A.dim() == 3 and A.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor of shape (w, n, lda)")


def _check_vec(v: torch.Tensor, name: str, n: Optional[int] = None):
    if not (v.is_cuda and v.dtype == torch.float64 and v.dim() == 2 and v.is_contiguous()
            and (n is None or v.shape[1] == n)):
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor of shape (w, n)"
                         + ("" if n is None else f" with n = {n}"))


# Every tensor below reaches the library as a raw device address with no
# extent attached, so the binding checks each one before any allocation or
# library call: a host tensor, another GPU's, the wrong element type or too
# few elements would otherwise become an out-of-bounds device access.

def _check_dev(t: torch.Tensor, name: str, device, dtype=torch.float64, numel: int = 0):
    """t: a contiguous CUDA tensor of `dtype` on `device` with at least
    `numel` elements."""
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous() and t.numel() >= numel
            and (device is None or t.device == device)):
        raise ValueError(f"{name} must be a contiguous {dtype} CUDA tensor on {device} "
                         f"with at least {numel} elements")


def _same_device(device, *named):
    for t, name in named:
        if t.device != device:
            raise ValueError(f"{name} is on {t.device}, the operands on {device}")


def _work_bytes(work: torch.Tensor, device) -> int:
    """A caller's work buffer (any element type): contiguous, on `device`;
    its size in bytes (the library checks it against what the call needs)."""
    if not (work.is_cuda and work.is_contiguous() and (device is None or work.device == device)):
        raise ValueError(f"work must be a contiguous CUDA tensor on {device}")
    return work.numel() * work.element_size()


def workspace(op: int, prec: int, update: int, n: int, device=None) -> torch.Tensor:
    nbytes = max(L.workspace_size(op, prec, update, n), 256)
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def ludecomp(A: torch.Tensor, prec="dd", update="plain", *, work: Optional[torch.Tensor] = None,
             stream=None, inplace: bool = False):
    """LU with partial pivoting (TDLUdecompPM).  Returns (LU, piv, info_tensor);
    LU has `prec` planes.  ``info`` is a device int64 tensor of one element
    (0, or k+1 for the first exactly zero pivot)."""
    _check_mat(A, "A")
    w = _prec(prec)
    u = UPDATE[update]
    n, lda = A.shape[1], A.shape[2]
    if work is not None:
        _work_bytes(work, A.device)
    if inplace:
        if A.shape[0] != w:
            raise ValueError("in-place factorisation needs exactly `prec` planes")
        LU = A
    else:
        LU = torch.zeros((w, n, lda), dtype=torch.float64, device=A.device)
        k = min(w, A.shape[0])
        LU[:k].copy_(A[:k])
    piv = torch.empty(max(n, 1), dtype=torch.int64, device=A.device)
    info = torch.zeros(1, dtype=torch.int64, device=A.device)
    if work is None:
        work = workspace(L.MW_OP_LUDECOMP, w, u, n, A.device)
    L.check("mw_ludecomp", L.lib().mw_ludecomp(w, u, n, _ptr(LU), lda, _ptr(piv), _ptr(info),
                                               _ptr(work), _work_bytes(work, A.device), _stream(stream)))
    return LU, piv[:n], info


def solve(LU: torch.Tensor, piv: torch.Tensor, b: torch.Tensor, prec=None, *,
          work: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None, stream=None):
    """Forward/back substitution (SolveTDLSPM).  b: (>=1, n); uses its first
    `prec` words (missing words are zero).  Returns x of shape (prec, n)."""
    _check_mat(LU, "LU")
    w = _prec(prec) if prec is not None else LU.shape[0]
    n, lda = LU.shape[1], LU.shape[2]
    if LU.shape[0] < w:
        raise ValueError("LU must hold at least `prec` planes")
    _check_dev(piv, "piv", LU.device, torch.int64, n)
    _check_vec(b, "b", n)
    _same_device(LU.device, (b, "b"))
    if out is not None:
        _check_dev(out, "out", LU.device, numel=w * n)
    if work is not None:
        _work_bytes(work, LU.device)
    if b.shape[0] != w:
        bb = torch.zeros((w, n), dtype=torch.float64, device=LU.device)
        k = min(w, b.shape[0])
        bb[:k].copy_(b[:k])
        b = bb
    x = out if out is not None else torch.empty((w, n), dtype=torch.float64, device=LU.device)
    if work is None:
        work = workspace(L.MW_OP_SOLVE, w, 0, n, LU.device)
    L.check("mw_solve", L.lib().mw_solve(w, n, _ptr(LU), lda, _ptr(piv), _ptr(b), _ptr(x),
                                         _ptr(work), _work_bytes(work, LU.device), _stream(stream)))
    return x


def residual(A: torch.Tensor, b: torch.Tensor, x: torch.Tensor, r_words: int = 8, *, stream=None,
             out: Optional[torch.Tensor] = None):
    """r = b - A x exactly, rounded greedily to r_words words."""
    _check_mat(A, "A")
    n, lda = A.shape[1], A.shape[2]
    _check_vec(b, "b", n)
    _check_vec(x, "x", n)
    _same_device(A.device, (b, "b"), (x, "x"))
    if out is not None:
        _check_dev(out, "out", A.device, numel=r_words * n)
    r = out if out is not None else torch.empty((r_words, n), dtype=torch.float64, device=A.device)
    L.check("mw_residual", L.lib().mw_residual(n, _ptr(A), lda, A.shape[0], _ptr(b), b.shape[0],
                                               _ptr(x), x.shape[0], _ptr(r), r_words, _stream(stream)))
    return r


@dataclass
class RefineResult:
    x: torch.Tensor
    status: int
    corrections: int
    residuals: int
    info: int

    @property
    def converged(self) -> bool:
        return self.status == L.MW_OK


def refine(A: torch.Tensor, b: torch.Tensor, inner_prec="td", target_bits: int = 200, *,
           update="plain", max_iter: int = 30, stop_mode: int = L.MW_STOP_BITS, rtol: float = 1e-100,
           atol: float = 0.0, x_words: int = 8, work: Optional[torch.Tensor] = None,
           out: Optional[torch.Tensor] = None, stream=None) -> RefineResult:
    """Mixed precision iterative refinement (Listing 1).  Returns a
    RefineResult; x has x_words planes (8 = 424 bits)."""
    _check_mat(A, "A")
    w = _prec(inner_prec)
    u = UPDATE[update]
    n, lda = A.shape[1], A.shape[2]
    _check_vec(b, "b", n)
    _same_device(A.device, (b, "b"))
    if out is not None:
        _check_dev(out, "out", A.device, numel=x_words * n)
    if work is not None:
        _work_bytes(work, A.device)
    x = out if out is not None else torch.empty((x_words, n), dtype=torch.float64, device=A.device)
    if work is None:
        work = workspace(L.MW_OP_REFINE, w, u, n, A.device)
    stats = (ctypes.c_int64 * 4)()
    rc = L.lib().mw_refine(n, _ptr(A), lda, A.shape[0], _ptr(b), b.shape[0], w, u, target_bits,
                           max_iter, stop_mode, rtol, atol, _ptr(x), x_words, stats, _ptr(work),
                           _work_bytes(work, A.device), _stream(stream))
    L.check("mw_refine", rc, ok=(L.MW_OK, L.MW_ENOTCONV, L.MW_ESINGULAR))
    return RefineResult(x, rc, int(stats[0]), int(stats[1]), int(stats[2]))


def _gemm(name: str, C, A, B, m, prec, update, work, stream):
    for t, nm in ((C, "C"), (A, "A"), (B, "B")):
        _check_mat(t, nm)
    _same_device(C.device, (A, "A"), (B, "B"))
    w = _prec(prec) if prec is not None else C.shape[0]
    u = UPDATE[update]
    N, ldc = C.shape[1], C.shape[2]
    K, lda = A.shape[1], A.shape[2]
    ldb = B.shape[2]
    if min(C.shape[0], A.shape[0], B.shape[0]) < w:
        raise ValueError("C, A and B must hold at least `prec` planes each")
    if B.shape[1] != N:
        raise ValueError("B must have the N columns of C: shape (w, N, ldb)")
    if work is not None:
        _work_bytes(work, C.device)
    if work is None:
        work = workspace(L.MW_OP_GEMM, w, u, max(m, N), C.device)
    L.check(name, getattr(L.lib(), name)(w, u, m, N, K, _ptr(C), ldc, _ptr(A), lda, _ptr(B), ldb,
                                         _ptr(work), _work_bytes(work, C.device), _stream(stream)))
    return C


def gemm_sub(C: torch.Tensor, A: torch.Tensor, B: torch.Tensor, m: int, prec=None, update="plain", *,
             work: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """C -= A B in multiword arithmetic on the leading m rows (in place;
    returns C).  C: (w, N, ldc), A: (w, K, lda), B: (w, N, ldb), component
    planes, column-major."""
    return _gemm("mw_gemm_sub", C, A, B, m, prec, update, work, stream)


def gemm_add(C: torch.Tensor, A: torch.Tensor, B: torch.Tensor, m: int, prec=None, update="plain", *,
             work: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """C += A B (the block matrix product; C = A B from a zero C), in place
    on the leading m rows; returns C.  Shapes as gemm_sub."""
    return _gemm("mw_gemm_add", C, A, B, m, prec, update, work, stream)


def gemm_strassen(A: torch.Tensor, B: torch.Tensor, prec=None, update="plain", levels: int = 1, *,
                  work: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None,
                  stream=None) -> torch.Tensor:
    """C = A B for n x n multiword matrices by Strassen's recursion over the
    block matrix product (`levels` levels).  A, B: (w, n, ld); returns C
    (w, n, n) (or `out`)."""
    _check_mat(A, "A")
    _check_mat(B, "B")
    w = _prec(prec) if prec is not None else A.shape[0]
    u = UPDATE[update]
    n = A.shape[1]
    if B.shape[1] != n or A.shape[0] < w or B.shape[0] < w:
        raise ValueError("A and B must be n x n with at least `prec` planes each")
    _same_device(A.device, (B, "B"))
    if out is not None:
        _same_device(A.device, (out, "out"))
    if work is not None:
        _work_bytes(work, A.device)
    if out is None:
        out = torch.empty((w, n, max(n, 1)), dtype=torch.float64, device=A.device)
    _check_mat(out, "out")
    if out.shape[0] < w or out.shape[1] != n or out.shape[2] < n:
        raise ValueError("out must hold `prec` planes of n x n")
    if work is None:
        nbytes = ctypes.c_size_t(0)
        L.check("mw_gemm_strassen_workspace_size",
                L.lib().mw_gemm_strassen_workspace_size(w, u, levels, n, ctypes.byref(nbytes)))
        work = torch.empty(max(int(nbytes.value), 256), dtype=torch.uint8, device=A.device)
    L.check("mw_gemm_strassen", L.lib().mw_gemm_strassen(w, u, levels, n, _ptr(A), A.shape[2], _ptr(B), B.shape[2],
                                                         _ptr(out), out.shape[2], _ptr(work),
                                                         _work_bytes(work, A.device), _stream(stream)))
    return out


def gemm(A: torch.Tensor, B: torch.Tensor, m: int, prec=None, update="plain", *,
         work: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """C = A B in multiword arithmetic: a new (w, N, m) tensor."""
    _check_mat(A, "A")
    _check_mat(B, "B")
    w = _prec(prec) if prec is not None else A.shape[0]
    if A.shape[0] < w or B.shape[0] < w:
        raise ValueError("A and B must hold at least `prec` planes each")
    _same_device(A.device, (B, "B"))
    C = torch.zeros((w, B.shape[1], max(m, 1)), dtype=torch.float64, device=A.device)
    return gemm_add(C, A, B, m, w, update, work=work, stream=stream)


# ---------------------------------------------------------------------------
# batches of independent systems (layout: include/mwlu.h, "Batches")
# ---------------------------------------------------------------------------

def batch_offsets(n_list):
    """(moff, voff) prefix offsets for the batch layout."""
    import numpy as np
    n = np.asarray(n_list, dtype=np.int64)
    moff = np.concatenate([[0], np.cumsum(n * n)])
    voff = np.concatenate([[0], np.cumsum(n)])
    return moff, voff


def pack_matrices(mats, w: int):
    """Pack a list of (>=1, n, lda) float64 arrays into the batch layout with
    w words per entry (missing words are zero).  Returns a numpy array."""
    import numpy as np
    n_list = [m.shape[1] for m in mats]
    moff, _ = batch_offsets(n_list)
    out = np.zeros(w * int(moff[-1]))
    for s, M in enumerate(mats):
        n = n_list[s]
        base = w * int(moff[s])
        for c in range(min(w, M.shape[0])):
            out[base + c * n * n: base + (c + 1) * n * n] = M[c, :, :n].reshape(-1)
    return out


def pack_vectors(vecs, w: int):
    import numpy as np
    n_list = [v.shape[1] for v in vecs]
    _, voff = batch_offsets(n_list)
    out = np.zeros(w * int(voff[-1]))
    for s, v in enumerate(vecs):
        n = n_list[s]
        base = w * int(voff[s])
        for c in range(min(w, v.shape[0])):
            out[base + c * n: base + (c + 1) * n] = v[c, :n]
    return out


def unpack_vectors(flat, n_list, w: int):
    import numpy as np
    _, voff = batch_offsets(n_list)
    return [np.asarray(flat[w * int(voff[s]): w * int(voff[s]) + w * n]).reshape(w, n)
            for s, n in enumerate(n_list)]


def unpack_matrices(flat, n_list, w: int):
    import numpy as np
    moff, _ = batch_offsets(n_list)
    return [np.asarray(flat[w * int(moff[s]): w * int(moff[s]) + w * n * n]).reshape(w, n, n)
            for s, n in enumerate(n_list)]


def _n_host(n_list):
    arr = (ctypes.c_int * len(n_list))(*[int(v) for v in n_list])
    return arr


def _batch_extent(n_list):
    """(sum of n, sum of n^2): the entries per word of the packed vectors and
    matrices (the library rejects orders outside its range itself)."""
    ns = [int(v) for v in n_list]
    return sum(ns), sum(v * v for v in ns)


def batch_workspace(op: int, prec: int, n_list, device=None) -> torch.Tensor:
    out = ctypes.c_size_t(0)
    L.check("mw_batch_workspace_size",
            L.lib().mw_batch_workspace_size(op, prec, len(n_list), _n_host(n_list), ctypes.byref(out)))
    return torch.empty(max(int(out.value), 256), dtype=torch.uint8, device=device or "cuda")


def ludecomp_batched(A: torch.Tensor, n_list, prec="dd", *, work=None, stream=None, inplace=False):
    """Batched LU (packed layout, `prec` words).  Returns (LU, piv, info)."""
    w = _prec(prec)
    _, sum_n2 = _batch_extent(n_list)
    _check_dev(A, "A", None, numel=w * sum_n2)
    if work is not None:
        _work_bytes(work, A.device)
    LU = A if inplace else A.clone()
    total_n = int(sum(n_list))
    piv = torch.empty(max(total_n, 1), dtype=torch.int64, device=A.device)
    info = torch.zeros(max(len(n_list), 1), dtype=torch.int64, device=A.device)
    if work is None:
        work = batch_workspace(L.MW_OP_LUDECOMP, w, n_list, A.device)
    L.check("mw_ludecomp_batched", L.lib().mw_ludecomp_batched(
        w, len(n_list), _n_host(n_list), _ptr(LU), _ptr(piv), _ptr(info), _ptr(work),
        _work_bytes(work, A.device), _stream(stream)))
    return LU, piv, info


def solve_batched(LU: torch.Tensor, piv: torch.Tensor, b: torch.Tensor, n_list, prec="dd", *, work=None,
                  out=None, stream=None):
    """Batched substitution: x (`prec` words per entry, packed like b) from
    the factors and pivots of ludecomp_batched or ludecomp_batched_blocked."""
    w = _prec(prec)
    sum_n, sum_n2 = _batch_extent(n_list)
    _check_dev(LU, "LU", None, numel=w * sum_n2)
    _check_dev(piv, "piv", LU.device, torch.int64, sum_n)
    _check_dev(b, "b", LU.device, numel=w * sum_n)
    if out is not None:
        _check_dev(out, "out", LU.device, numel=w * sum_n)
    if work is not None:
        _work_bytes(work, LU.device)
    x = out if out is not None else torch.empty_like(b)
    if work is None:
        work = batch_workspace(L.MW_OP_SOLVE, w, n_list, LU.device)
    L.check("mw_solve_batched", L.lib().mw_solve_batched(
        w, len(n_list), _n_host(n_list), _ptr(LU), _ptr(piv), _ptr(b), _ptr(x), _ptr(work),
        _work_bytes(work, LU.device), _stream(stream)))
    return x


def refine_batched(A: torch.Tensor, a_words: int, b: torch.Tensor, b_words: int, n_list, inner_prec="dd",
                   target_bits: int = 200, *, max_iter: int = 30, x_words: int = 8, work=None, out=None,
                   stream=None):
    """Batched refinement; returns (x, stats) with stats an int64 tensor
    (count, 4): corrections, residuals, LU info, status."""
    w = _prec(inner_prec)
    total_n, sum_n2 = _batch_extent(n_list)
    _check_batch_refine(A, a_words, b, b_words, x_words, total_n, sum_n2, out, work)
    x = out if out is not None else torch.empty(x_words * total_n, dtype=torch.float64, device=A.device)
    stats = torch.zeros((len(n_list), 4), dtype=torch.int64, device=A.device)
    if work is None:
        work = batch_workspace(L.MW_OP_REFINE, w, n_list, A.device)
    L.check("mw_refine_batched", L.lib().mw_refine_batched(
        len(n_list), _n_host(n_list), _ptr(A), a_words, _ptr(b), b_words, w, target_bits, max_iter, _ptr(x),
        x_words, _ptr(stats), _ptr(work), _work_bytes(work, A.device), _stream(stream)))
    return x, stats


def _check_batch_refine(A, a_words, b, b_words, x_words, total_n, sum_n2, out, work):
    if min(a_words, b_words, x_words) < 1:
        raise ValueError("a_words, b_words and x_words must be at least 1")
    _check_dev(A, "A", None, numel=a_words * sum_n2)
    _check_dev(b, "b", A.device, numel=b_words * total_n)
    if out is not None:
        _check_dev(out, "out", A.device, numel=x_words * total_n)
    if work is not None:
        _work_bytes(work, A.device)


def _update(update) -> int:
    if update in ("plain", L.MW_UPDATE_PLAIN):
        return L.MW_UPDATE_PLAIN
    if update in ("split", L.MW_UPDATE_SPLIT):
        return L.MW_UPDATE_SPLIT
    raise ValueError(f"update must be 'plain' or 'split', not {update!r}")


def batch_blocked_workspace(op: int, prec: int, update, n_list, device=None) -> torch.Tensor:
    out = ctypes.c_size_t(0)
    L.check("mw_batch_blocked_workspace_size",
            L.lib().mw_batch_blocked_workspace_size(op, prec, _update(update), len(n_list), _n_host(n_list),
                                                    ctypes.byref(out)))
    return torch.empty(max(int(out.value), 256), dtype=torch.uint8, device=device or "cuda")


def ludecomp_batched_blocked(A: torch.Tensor, n_list, prec="dd", update="plain", *, work=None, stream=None,
                             inplace=False):
    """Blocked batched LU (packed layout): all systems advance one 64-column
    panel per step; the trailing update of every active system is one launch
    (plain multiword GEMM or, for DD, the split tensor-core form).
    Returns (LU, piv, info)."""
    w = _prec(prec)
    u = _update(update)
    _, sum_n2 = _batch_extent(n_list)
    _check_dev(A, "A", None, numel=w * sum_n2)
    if work is not None:
        _work_bytes(work, A.device)
    LU = A if inplace else A.clone()
    total_n = int(sum(n_list))
    piv = torch.empty(max(total_n, 1), dtype=torch.int64, device=A.device)
    info = torch.zeros(max(len(n_list), 1), dtype=torch.int64, device=A.device)
    if work is None:
        work = batch_blocked_workspace(L.MW_OP_LUDECOMP, w, u, n_list, A.device)
    L.check("mw_ludecomp_batched_blocked", L.lib().mw_ludecomp_batched_blocked(
        w, u, len(n_list), _n_host(n_list), _ptr(LU), _ptr(piv), _ptr(info), _ptr(work),
        _work_bytes(work, A.device), _stream(stream)))
    return LU, piv, info


def refine_batched_blocked(A: torch.Tensor, a_words: int, b: torch.Tensor, b_words: int, n_list,
                           inner_prec="dd", update="split", target_bits: int = 200, *, max_iter: int = 30,
                           x_words: int = 8, work=None, out=None, stream=None):
    """refine_batched with the inner LU factored by the blocked batched LU."""
    w = _prec(inner_prec)
    u = _update(update)
    total_n, sum_n2 = _batch_extent(n_list)
    _check_batch_refine(A, a_words, b, b_words, x_words, total_n, sum_n2, out, work)
    x = out if out is not None else torch.empty(x_words * total_n, dtype=torch.float64, device=A.device)
    stats = torch.zeros((len(n_list), 4), dtype=torch.int64, device=A.device)
    if work is None:
        work = batch_blocked_workspace(L.MW_OP_REFINE, w, u, n_list, A.device)
    L.check("mw_refine_batched_blocked", L.lib().mw_refine_batched_blocked(
        len(n_list), _n_host(n_list), _ptr(A), a_words, _ptr(b), b_words, w, u, target_bits, max_iter,
        _ptr(x), x_words, _ptr(stats), _ptr(work), _work_bytes(work, A.device), _stream(stream)))
    return x, stats


def batch_plan_cache(on: bool) -> bool:
    """Switch the record of resident batch plans on or off (off forgets all);
    returns the previous setting.  With it on, repeated batched LU / solve
    calls on the same batch and work buffers upload nothing and can be
    captured in a CUDA graph; keep those work buffers alive meanwhile."""
    return bool(L.lib().mw_batch_plan_cache(1 if on else 0))


def arith(op: int, prec, x: torch.Tensor, y: torch.Tensor, *, stream=None) -> torch.Tensor:
    """Element-wise multiword op (0 add, 1 sub, 2 mul, 3 div, 4 compare |x|,|y|)."""
    w = _prec(prec)
    _check_vec(x, "x")
    _check_vec(y, "y")
    if y.shape != x.shape or x.shape[0] < w:
        raise ValueError("x and y must have the same shape (planes >= prec, cnt)")
    _same_device(x.device, (y, "y"))
    z = torch.empty_like(x)
    L.check("mw_arith", L.lib().mw_arith(op, w, x.shape[1], _ptr(x), _ptr(y), _ptr(z), _stream(stream)))
    return z


def peak_fp64() -> float:
    """FP64 instructions per second measured by the library's microbenchmark."""
    out = ctypes.c_double(0.0)
    L.check("mw_peak_fp64", L.lib().mw_peak_fp64(ctypes.byref(out), _stream()))
    return out.value


def work_status(op: int, update, work: torch.Tensor, *, stream=None) -> int:
    """MW_OK or MW_ETIMEOUT for the last call that used this single-system
    work buffer (synchronises the stream; mw_work_status)."""
    _work_bytes(work, None)
    return L.check("mw_work_status", L.lib().mw_work_status(op, UPDATE[update], _ptr(work), _stream(stream)),
                   ok=(L.MW_OK, L.MW_ETIMEOUT))


def batch_work_status(work: torch.Tensor, *, stream=None) -> int:
    """MW_OK or MW_ETIMEOUT for the last batched call that used this work
    buffer (synchronises the stream; mw_batch_work_status)."""
    _work_bytes(work, None)
    return L.check("mw_batch_work_status", L.lib().mw_batch_work_status(_ptr(work), _stream(stream)),
                   ok=(L.MW_OK, L.MW_ETIMEOUT))


def set_wait_limit(polls: int) -> int:
    """Poll limit of the bounded device waits for later launches (0: each
    kernel's default); returns the previous value (mw_set_wait_limit)."""
    prev = int(L.lib().mw_set_wait_limit(int(polls)))
    if prev < 0:
        raise ValueError("polls must be >= 0")
    return prev
