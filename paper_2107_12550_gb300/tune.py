"""Autotuner for the library's blocking knobs, with a JSON cache.

The knobs (``include/mwlu.h``, MW_TUNE_*) change only the blocking: the
panel width of the plain blocked LU, the panel rows per CTA, and the
persistent CTAs per SM of the batched LU.  Results are bitwise the same for
every value, so tuning is purely a speed choice.  The tuner times the
candidates through the public API on synthetic inputs of the requested size,
keeps the fastest, and stores it in a JSON cache keyed by GPU name,
precision, operation and size bucket (``MWLU_TUNE_CACHE``, default
``~/.cache/mwlu/tune.json``).  ``apply`` sets the knobs from the cache.
"""
from __future__ import annotations

import json
import math
import os
import time
from typing import Callable, Dict, Iterable, Optional

from . import _lib as L

PANEL_WIDTHS = (32, 64, 128)
ROWS_PER_CTA = (4, 8, 16, 32)
BATCH_CTAS = (1, 2, 3, 4)


def cache_path() -> str:
    return os.environ.get("MWLU_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "mwlu", "tune.json"))


def bucket(n: int) -> int:
    """Size bucket: n rounded up to a power of two (at least 16)."""
    return 1 << max(4, int(math.ceil(math.log2(max(n, 1)))))


def key(gpu: str, prec: int, op: str, n: int) -> str:
    return f"{gpu}|w{prec}|{op}|{bucket(n)}"


def load_cache(path: Optional[str] = None) -> Dict[str, dict]:
    path = path or cache_path()
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save_cache(cache: Dict[str, dict], path: Optional[str] = None) -> None:
    path = path or cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def pick_best(candidates: Iterable, timer: Callable[[object], float]) -> tuple:
    """(best candidate, {candidate: seconds}) by calling timer(candidate)."""
    times = {}
    for c in candidates:
        times[c] = timer(c)
    best = min(times, key=times.get)
    return best, times


def set_knob(param: int, prec: int, value: int) -> int:
    prev = L.lib().mw_set_tuning(param, prec, value)
    if prev < 0:
        raise ValueError(f"mw_set_tuning({param}, {prec}, {value}) -> {prev}")
    return prev


def _gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def tune_lu(prec: int, n: int, *, reps: int = 1, path: Optional[str] = None, widths=PANEL_WIDTHS,
            rows=ROWS_PER_CTA) -> dict:
    """Time the plain LU of a uniform n x n matrix over panel widths and rows
    per CTA; store and apply the fastest."""
    import torch
    from . import api, workloads as W
    A = torch.from_numpy(W.uniform_matrix(n, prec, seed=12345)).cuda()
    work = api.workspace(L.MW_OP_LUDECOMP, prec, 0, n)

    def timer(cand):
        nb, rpc = cand
        set_knob(L.MW_TUNE_PANEL_WIDTH, prec, nb)
        set_knob(L.MW_TUNE_PANEL_ROWS_PER_CTA, prec, rpc)
        api.ludecomp(A, prec, work=work)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            api.ludecomp(A, prec, work=work)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    best, times = pick_best([(w, r) for w in widths for r in rows], timer)
    entry = {"panel_width": best[0], "rows_per_cta": best[1],
             "seconds": {f"{w}x{r}": t for (w, r), t in times.items()}}
    cache = load_cache(path)
    cache[key(_gpu_name(), prec, "lu", n)] = entry
    save_cache(cache, path)
    set_knob(L.MW_TUNE_PANEL_WIDTH, prec, best[0])
    set_knob(L.MW_TUNE_PANEL_ROWS_PER_CTA, prec, best[1])
    return entry


def tune_batched(prec: int, n_list, *, reps: int = 1, path: Optional[str] = None, ctas=BATCH_CTAS) -> dict:
    """Time the batched LU over persistent CTAs per SM; store and apply the fastest."""
    import torch
    from . import api, workloads as W
    mats = [W.uniform_matrix(int(m), prec, seed=W.system_seed(7, s), lda=int(m)) for s, m in enumerate(n_list)]
    A = torch.from_numpy(api.pack_matrices(mats, prec)).cuda()
    work = api.batch_workspace(L.MW_OP_LUDECOMP, prec, n_list)
    LU = torch.empty_like(A)

    def timer(c):
        set_knob(L.MW_TUNE_BATCH_CTAS_PER_SM, prec, c)
        LU.copy_(A)
        api.ludecomp_batched(LU, n_list, prec, work=work, inplace=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            LU.copy_(A)
            api.ludecomp_batched(LU, n_list, prec, work=work, inplace=True)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps

    best, times = pick_best(ctas, timer)
    entry = {"ctas_per_sm": best, "seconds": {str(c): t for c, t in times.items()}}
    cache = load_cache(path)
    cache[key(_gpu_name(), prec, "batched", max(n_list))] = entry
    save_cache(cache, path)
    set_knob(L.MW_TUNE_BATCH_CTAS_PER_SM, prec, best)
    return entry


def apply(prec: int, n: int, *, op: str = "lu", path: Optional[str] = None, gpu: Optional[str] = None) -> bool:
    """Set the knobs from the cache for (gpu, prec, op, bucket(n)); False if
    there is no entry."""
    cache = load_cache(path)
    e = cache.get(key(gpu or _gpu_name(), prec, op, n))
    if not e:
        return False
    if op == "lu":
        set_knob(L.MW_TUNE_PANEL_WIDTH, prec, int(e["panel_width"]))
        set_knob(L.MW_TUNE_PANEL_ROWS_PER_CTA, prec, int(e["rows_per_cta"]))
    else:
        set_knob(L.MW_TUNE_BATCH_CTAS_PER_SM, prec, int(e["ctas_per_sm"]))
    return True
