"""Autotuner for the library's blocking knobs, with a JSON cache.

The knobs (``include/mwlu.h``, MW_TUNE_*) change only the blocking:
* plain LU (op "lu"): the panel width and the panel rows per CTA (results
  bitwise the same for every value);
* split LU of one system (op "split_lu"): the recursive panel's leaf width
  and the panel rows per CTA (roundings only, within the split path's bound);
* blocked batched split LU (op "batched_split"): the recursive panel's leaf
  width;
* persistent batched LU (op "batched"): CTAs per SM.
The tuner times the candidates through the public API on synthetic inputs of
the requested size, keeps the fastest, and stores it in a JSON cache keyed
by GPU name, precision, operation and size bucket.  The cache is the user's
file (``MWLU_TUNE_CACHE``, default ``~/.cache/mwlu/tune.json``) over the
table measured on GB300 that ships with the package (``tune_gb300.json``).
``apply`` sets the knobs from the cache.  ``python -m
paper_2107_12550_gb300.tune --out FILE`` measures the standard set.
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
SPLIT_LEAVES = (0, 8, 16, 32)        # 0: no recursion below the 64-column panel
BATCH_SPLIT_LEAVES = (8, 16, 32)
PACKAGED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_gb300.json")


def cache_path() -> str:
    return os.environ.get("MWLU_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "mwlu", "tune.json"))


def bucket(n: int) -> int:
    """Size bucket: n rounded up to a power of two (at least 16)."""
    return 1 << max(4, int(math.ceil(math.log2(max(n, 1)))))


def key(gpu: str, prec: int, op: str, n: int) -> str:
    return f"{gpu}|w{prec}|{op}|{bucket(n)}"


def _read(path: str) -> Dict[str, dict]:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def load_cache(path: Optional[str] = None) -> Dict[str, dict]:
    """The given cache file; without one, the packaged GB300 table overlaid
    with the user's cache."""
    if path:
        return _read(path)
    merged = _read(PACKAGED)
    merged.update(_read(cache_path()))
    return merged


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
    _store(prec, "lu", n, entry, path)
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
    _store(prec, "batched", max(n_list), entry, path)
    set_knob(L.MW_TUNE_BATCH_CTAS_PER_SM, prec, best)
    return entry


def _store(prec: int, op: str, n: int, entry: dict, path: Optional[str]) -> None:
    target = path or cache_path()
    cache = _read(target)
    cache[key(_gpu_name(), prec, op, n)] = entry
    save_cache(cache, target)


def _time_calls(fn, reps: int) -> float:
    import torch
    fn()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        fn()
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / reps


def tune_split_lu(n: int, *, reps: int = 2, path: Optional[str] = None, leaves=SPLIT_LEAVES,
                  rows=(4, 8, 16)) -> dict:
    """Time the split DD LU of a uniform n x n matrix over the recursive
    panel's leaf widths and the panel rows per CTA; store and apply the
    fastest."""
    import torch
    from . import api, workloads as W
    A = torch.from_numpy(W.uniform_matrix(n, 2, seed=12345)).cuda()
    work = api.workspace(L.MW_OP_LUDECOMP, 2, 1, n)

    def timer(cand):
        leaf, rpc = cand
        set_knob(L.MW_TUNE_SPLIT_PANEL_LEAF, 2, leaf)
        set_knob(L.MW_TUNE_PANEL_ROWS_PER_CTA, 2, rpc)
        return _time_calls(lambda: api.ludecomp(A, 2, "split", work=work), reps)

    best, times = pick_best([(lf, r) for lf in leaves for r in rows], timer)
    entry = {"split_leaf": best[0], "rows_per_cta": best[1],
             "seconds": {f"{lf}x{r}": t for (lf, r), t in times.items()}}
    _store(2, "split_lu", n, entry, path)
    set_knob(L.MW_TUNE_SPLIT_PANEL_LEAF, 2, best[0])
    set_knob(L.MW_TUNE_PANEL_ROWS_PER_CTA, 2, best[1])
    return entry


def tune_batched_split(n_list, *, reps: int = 2, path: Optional[str] = None, leaves=BATCH_SPLIT_LEAVES) -> dict:
    """Time the blocked batched split DD LU of a batch of uniform matrices
    with the given orders over the recursive panel's leaf widths; store
    (keyed by the largest order) and apply the fastest."""
    import torch
    from . import api, workloads as W
    mats = [W.uniform_matrix(int(m), 2, seed=W.system_seed(11, s), lda=int(m)) for s, m in enumerate(n_list)]
    A = torch.from_numpy(api.pack_matrices(mats, 2)).cuda()
    del mats
    work = api.batch_blocked_workspace(L.MW_OP_LUDECOMP, 2, "split", n_list)
    LU = torch.empty_like(A)

    def run():
        LU.copy_(A)
        api.ludecomp_batched_blocked(LU, n_list, 2, "split", work=work, inplace=True)

    def timer(leaf):
        set_knob(L.MW_TUNE_BATCH_SPLIT_LEAF, 2, leaf)
        return _time_calls(run, reps)

    best, times = pick_best(leaves, timer)
    entry = {"batch_split_leaf": best, "seconds": {str(c): t for c, t in times.items()}}
    _store(2, "batched_split", max(n_list), entry, path)
    set_knob(L.MW_TUNE_BATCH_SPLIT_LEAF, 2, best)
    return entry


KNOBS = {
    "lu": (("panel_width", L.MW_TUNE_PANEL_WIDTH), ("rows_per_cta", L.MW_TUNE_PANEL_ROWS_PER_CTA)),
    "split_lu": (("split_leaf", L.MW_TUNE_SPLIT_PANEL_LEAF), ("rows_per_cta", L.MW_TUNE_PANEL_ROWS_PER_CTA)),
    "batched_split": (("batch_split_leaf", L.MW_TUNE_BATCH_SPLIT_LEAF),),
    "batched": (("ctas_per_sm", L.MW_TUNE_BATCH_CTAS_PER_SM),),
}


def apply(prec: int, n: int, *, op: str = "lu", path: Optional[str] = None, gpu: Optional[str] = None):
    """Set the knobs from the cache for (gpu, prec, op, bucket(n)); returns
    the applied {knob: value}, or None if there is no entry."""
    cache = load_cache(path)
    e = cache.get(key(gpu or _gpu_name(), prec, op, n))
    if not e:
        return None
    applied = {}
    for name, param in KNOBS[op]:
        if name in e:
            set_knob(param, prec, int(e[name]))
            applied[name] = int(e[name])
    return applied


def main(argv=None) -> int:
    """Measure the standard set on this GPU and write it to --out: the plain
    TD LU at n = 2048, the split DD LU at n = 4096 and 8192, the blocked
    batched split LU of 512 orders uniform in [64, 1024], and the persistent
    batched LU of 4096 orders uniform in [16, 256] (DD and TD)."""
    import argparse
    from . import build, workloads as W
    p = argparse.ArgumentParser()
    p.add_argument("--out", required=True)
    a = p.parse_args(argv)
    build.build()
    print("lu td 2048", tune_lu(3, 2048, path=a.out), flush=True)
    for n in (4096, 8192):
        print("split_lu dd", n, tune_split_lu(n, reps=1 if n > 4096 else 2, path=a.out), flush=True)
    n_list, _ = W.mixed_batch_spec(512, 64, 1024, 4.0, 20.0, seed=0)
    print("batched_split dd", tune_batched_split(n_list, path=a.out), flush=True)
    small = [int(v) for v in W.batch_sizes(4096, 16, 256, seed=0)]
    for w in (2, 3):
        print("batched", w, tune_batched(w, small, path=a.out), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
