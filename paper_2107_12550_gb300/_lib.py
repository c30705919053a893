"""ctypes loader for libmwlu.so (the library's C ABI, ``include/mwlu.h``).

The product path has no fallback: if the library is missing or fails to
load, every call raises.  Build it with ``paper_2107_12550_gb300.build.build()``.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmwlu.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "mwlu.h")

MW_DD, MW_TD, MW_QD, MW_LONG_WORDS = 2, 3, 4, 8
MW_UPDATE_PLAIN, MW_UPDATE_SPLIT = 0, 1
MW_OK, MW_ESINGULAR, MW_ENOTCONV, MW_ECUDA, MW_ETIMEOUT, MW_EUNSUPPORTED = 0, 1, 2, 3, 4, 5
MW_OP_LUDECOMP, MW_OP_SOLVE, MW_OP_REFINE, MW_OP_GEMM = 0, 1, 2, 3
MW_STOP_EQ2, MW_STOP_BITS = 0, 1
MW_TUNE_PANEL_WIDTH, MW_TUNE_PANEL_ROWS_PER_CTA, MW_TUNE_BATCH_CTAS_PER_SM = 0, 1, 2
MW_TUNE_SPLIT_PANEL_LEAF = 3
MW_TUNE_GEMM_TILE = 4
MW_TUNE_BATCH_SPLIT_LEAF = 5
MW_TUNE_LOOKAHEAD = 6

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_D = ctypes.c_double
_SZ = ctypes.c_size_t

SIGNATURES = {
    "mw_workspace_size": (_I, [_I, _I, _I, _I64, ctypes.POINTER(_SZ)]),
    "mw_ludecomp": (_I, [_I, _I, _I64, _P, _I64, _P, _P, _P, _SZ, _P]),
    "mw_solve": (_I, [_I, _I64, _P, _I64, _P, _P, _P, _P, _SZ, _P]),
    "mw_residual": (_I, [_I64, _P, _I64, _I, _P, _I, _P, _I, _P, _I, _P]),
    "mw_refine": (_I, [_I64, _P, _I64, _I, _P, _I, _I, _I, _I, _I, _I, _D, _D, _P, _I, _P, _P, _SZ, _P]),
    "mw_arith": (_I, [_I, _I, _I64, _P, _P, _P, _P]),
    "mw_gemm_sub": (_I, [_I, _I, _I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _SZ, _P]),
    "mw_gemm_add": (_I, [_I, _I, _I64, _I64, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _SZ, _P]),
    "mw_gemm_strassen_workspace_size": (_I, [_I, _I, _I, _I64, _P]),
    "mw_gemm_strassen": (_I, [_I, _I, _I, _I64, _P, _I64, _P, _I64, _P, _I64, _P, _SZ, _P]),
    "mw_peak_fp64": (_I, [ctypes.POINTER(_D), _P]),
    "mw_solve_noalloc": (_I, [_I, _I64, _P, _I64, _P, _P, _P, _P]),
    "mw_batch_workspace_size": (_I, [_I, _I, _I, _P, ctypes.POINTER(_SZ)]),
    "mw_ludecomp_batched": (_I, [_I, _I, _P, _P, _P, _P, _P, _SZ, _P]),
    "mw_solve_batched": (_I, [_I, _I, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "mw_refine_batched": (_I, [_I, _P, _P, _I, _P, _I, _I, _I, _I, _P, _I, _P, _P, _SZ, _P]),
    "mw_batch_blocked_workspace_size": (_I, [_I, _I, _I, _I, _P, ctypes.POINTER(_SZ)]),
    "mw_ludecomp_batched_blocked": (_I, [_I, _I, _I, _P, _P, _P, _P, _P, _SZ, _P]),
    "mw_refine_batched_blocked": (_I, [_I, _P, _P, _I, _P, _I, _I, _I, _I, _I, _P, _I, _P, _P, _SZ, _P]),
    "mw_batch_plan_cache": (_I, [_I]),
    "mw_batch_plan_reset": (_I, []),
    "mw_profile_enable": (_I, [_I]),
    "mw_profile_read": (_I, [ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong), _I, _I]),
    "mw_set_tuning": (_I, [_I, _I, _I]),
    "mw_get_tuning": (_I, [_I, _I]),
    "mw_strerror": (ctypes.c_char_p, [_I]),
    "mw_last_cuda_error": (_I, []),
    "mw_version": (ctypes.c_char_p, []),
    "mw_work_status": (_I, [_I, _I, _P, _P]),
    "mw_batch_work_status": (_I, [_P, _P]),
    "mw_solve_noalloc_status": (_I, [_P]),
    "mw_set_wait_limit": (ctypes.c_longlong, [ctypes.c_longlong]),
}

_lock = threading.Lock()
_lib = None


class MWError(RuntimeError):
    def __init__(self, fn: str, code: int):
        self.code = code
        msg = lib().mw_strerror(code).decode() if _lib is not None else str(code)
        extra = ""
        if code == MW_ECUDA:
            extra = f" (cudaError {lib().mw_last_cuda_error()})"
        super().__init__(f"{fn} returned {code}: {msg}{extra}")


def lib() -> ctypes.CDLL:
    """Load libmwlu.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with paper_2107_12550_gb300.build.build() "
                    "(there is no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def check(fn: str, code: int, ok=(MW_OK,)) -> int:
    if code not in ok:
        raise MWError(fn, code)
    return code


def workspace_size(op: int, prec: int, update: int, n: int) -> int:
    out = _SZ(0)
    check("mw_workspace_size", lib().mw_workspace_size(op, prec, update, n, ctypes.byref(out)))
    return int(out.value)


PHASES = ["panel", "laswp", "trsm", "gemm_plain", "gemm_split", "solve", "perm", "residual",
          "refine_aux", "split_aux", "batch_lu", "batch_solve", "panel_inner"]


def profile_enable(on: bool = True) -> None:
    check("mw_profile_enable", lib().mw_profile_enable(1 if on else 0))


def profile_read(reset: bool = True) -> dict:
    """{phase: (ms, launches)} for the library's launches since the last reset."""
    n = len(PHASES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_longlong * n)()
    check("mw_profile_read", lib().mw_profile_read(ms, cnt, n, 1 if reset else 0))
    return {p: (ms[i], int(cnt[i])) for i, p in enumerate(PHASES)}


def declared_symbols() -> list:
    """Names of the functions declared in include/mwlu.h."""
    import re
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:int|long long|const char\*)\s+(mw_\w+)\s*\(", text, re.M)))
