#!/usr/bin/env python3
"""Benchmark of the multiword direct solver + mixed precision iterative
refinement (Kouya, arXiv 2107.12550, Section 2 Listing 1 and Section 3).

Headline workload (one GPU): a batch of 512 independent dense systems,
n_i uniform in [64, 1024], condition numbers log-uniform in [1e4, 1e20];
each A_i = U diag(sigma) V^T with U, V Haar-orthogonal (Householder QR of
Gaussian matrices, quantised to 2^-20) and sigma geometric from 1 to 1/kappa_i
(powers of two), stored exactly in QD (4 words); b_i = A_i * ones exactly in
8 words, so x* = ones.  A step is one replay of a CUDA graph holding one call
of the library's blocked batched refinement (captured once; its refinement
loop is a graph while node whose condition the device sets): the DD LU of every system with the split-precision (bf16
tensor-core Ozaki) trailing update, the DD substitution, and per system the
loop r = b - A x (exact, rounded to 8 words = 424 bits), z = solve(2^-e r),
x = RN_8(x + 2^e z) until the correction is below 2^-202 ||x||.  Metric:
systems solved to 2^-200 relative forward error per second, from
device-resident (A, b) to device-resident x.  The plain FP64-core forms (the
same batch with the plain DD LU; one n = 2048 system with the plain TD LU)
are reported beside it.

Multi-GPU: every rank solves its own independent batch (seeded by rank), no
collective on the data path (weak scaling); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time
from fractions import Fraction

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

TARGET_BITS = 200
X_WORDS = 8
# the headline batch
BATCH = 512
N_LO, N_HI = 64, 1024
LOG10_KAPPA_LO, LOG10_KAPPA_HI = 4.0, 20.0
A_WORDS = 4


def workload_name(count: int) -> str:
    return (f"mixed_batch_{count}_svd_n{N_LO}-{N_HI}_kappa1e{LOG10_KAPPA_LO:g}-1e{LOG10_KAPPA_HI:g}"
            f"_qd_stored_split_dd_inner_refine_to_2^-{TARGET_BITS}")


# the single-system comparator (plain TD LU)
N = 2048
LOG10_KAPPA = 10.0
INNER = 3                 # TD

# FP64 instructions of one multiword multiply + subtraction (the elimination
# step), counted from the algorithms in csrc/mw_arith.cuh on their typical
# (all error terms non-zero) path: with TwoSum's FP64 sequence (the serial
# chains: single-system panel, TRSM and solve, the substitution's leader) and
# with TwoSum on the integer pipes (the throughput loops: the GEMMs, the
# batched panel leaves, the substitution's workers), where each TwoSum's six
# FP64 instructions leave the FP64 pipe
FP64_PER_MSUB = {2: 29, 3: 117, 4: 196}
FP64_PER_MSUB_INT = {2: 17, 3: 27, 4: 46}
# FP64 thread instructions per clock of the whole GB300 (ncu: the
# peak_sustained of sm__sass_thread_inst_executed_op_dfma_pred_on.sum,
# 2 per SM per clock over 152 SMs)
FP64_LANES_PER_CLK = 304
# bf16 MMA flops of one 128 x 16 output tile of the split update: 120 digit
# pairs x 2 x 128 x 16 x 64
SPLIT_TILE_FLOPS = 120 * 2 * 128 * 16 * 64

# DRAM bytes (read + write) per launch of the TD plain trailing update in the
# n = 2048 single-system workload with the packaged tuning (panel 32 x 16
# rows; with the look-ahead, two update launches per panel step): ncu
# dram__bytes_read.sum + dram__bytes_write.sum over the LU's 125 launches
# (2266.1 + 234.5 MB), averaged per launch.  Must be re-measured whenever
# k_gemm_plain changes.
GEMM_TD_TRAFFIC_PER_LAUNCH = 20.0e6
# DRAM bytes per multiword multiply-subtract of the batched substitution:
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_solve_batched<DD>
# launch (the second solve of the 152-system mixed batch, n <= 1024, all 152
# systems running: 1033.9 + 3.9 MB) over its sum of n^2 (59.08 M); the
# algorithmic figure is 16 bytes (each DD entry of L and U read once).  Must
# be re-measured whenever k_solve_batched changes.
SOLVE_BATCHED_TRAFFIC_PER_MSUB = 1037.8e6 / 59.08e6

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="mwlu", choices=["mwlu", "reference"])
    p.add_argument("--count", type=int, default=BATCH, help="systems in the headline batch")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the comparison measurements (plain forms, large LU, standalone GEMM, batches)")
    return p.parse_args()


def measured_peaks() -> dict:
    """The measured peaks of this GPU pool (MEASURED_PEAKS.json next to
    this file), or {} when absent."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled during the timed region."""

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={CLOCK_FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def combine_ranks(ms: float, solved: int, device) -> tuple:
    """(max time over the ranks, systems solved by all ranks) across the
    process group; the rank's own values without one (replicas: no data
    leaves a rank, only these two numbers)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms, solved
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    c = torch.tensor([float(solved)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t[0]), int(c[0])


def exact_ok(x_host, n) -> bool:
    """|x_i - 1| <= 2^-200 for every i, evaluated exactly on the words."""
    lim = Fraction(1, 2 ** TARGET_BITS)
    for i in range(n):
        v = sum((Fraction(float(x_host[c, i])) for c in range(x_host.shape[0])), Fraction(0))
        if abs(v - 1) > lim:
            return False
    return True


def panel_sum_sq(n: int, nb: int = 64) -> int:
    """sum over panels of (rows below) x (cols right) x nb: multiword
    multiply-subtract steps of the trailing updates."""
    tot = 0
    for k0 in range(0, n, nb):
        kb = min(nb, n - k0)
        r = n - k0 - kb
        tot += r * r * kb
    return tot




DEFAULT_KNOBS = {"panel_width": 64, "rows_per_cta": 8, "ctas_per_sm": 2, "split_leaf": 0, "gemm_tile": 0,
                 "batch_split_leaf": 8, "lookahead": 1}


def reset_knobs():
    """Every tuning knob back to the library's default, for every precision."""
    from paper_2107_12550_gb300 import _lib as L
    params = {"panel_width": L.MW_TUNE_PANEL_WIDTH, "rows_per_cta": L.MW_TUNE_PANEL_ROWS_PER_CTA,
              "ctas_per_sm": L.MW_TUNE_BATCH_CTAS_PER_SM, "split_leaf": L.MW_TUNE_SPLIT_PANEL_LEAF,
              "gemm_tile": L.MW_TUNE_GEMM_TILE, "batch_split_leaf": L.MW_TUNE_BATCH_SPLIT_LEAF,
              "lookahead": L.MW_TUNE_LOOKAHEAD}
    for name, prm in params.items():
        for w in (2, 3, 4):
            L.lib().mw_set_tuning(prm, w, DEFAULT_KNOBS[name])


def tuned(prec: int, n: int, op: str) -> dict:
    """The knobs of the tuning cache (the packaged GB300 table under the
    user's cache) for this operation and size, applied over the defaults;
    {} when the cache has no entry."""
    from paper_2107_12550_gb300 import tune as T
    reset_knobs()
    return T.apply(prec, n, op=op) or {}


def split_trail_mma_flops(n_list, nb: int = 64) -> int:
    """bf16 MMA flops of the trailing split updates of one blocked batched
    LU: per panel step and active system, ceil(m / 128) x ceil(m / 16) tiles
    of the m x m trailing block, each SPLIT_TILE_FLOPS."""
    tiles = 0
    for n in n_list:
        for k0 in range(0, n, nb):
            m = n - k0 - nb
            if m > 0:
                tiles += (-(-m // 128)) * (-(-m // 16))
    return tiles * SPLIT_TILE_FLOPS


def batch_system(A_np, b_np, n_list, s, a_words=A_WORDS, b_words=X_WORDS):
    """System s of a packed batch as the oracle's (w, n, n) matrix and (w, n) vector."""
    import numpy as np
    n = n_list[s]
    moff = int(sum(m * m for m in n_list[:s]))
    voff = int(sum(n_list[:s]))
    A = np.ascontiguousarray(A_np[a_words * moff: a_words * (moff + n * n)].reshape(a_words, n, n))
    b = np.ascontiguousarray(b_np[b_words * voff: b_words * (voff + n)].reshape(b_words, n))
    return A, b


def stratified_sample(n_list, stride: int):
    """Every stride-th system in order of n (ties by index): a sample whose
    mix of orders follows the batch's."""
    order = sorted(range(len(n_list)), key=lambda s: (n_list[s], s))
    return order[stride // 2::stride]


def oracle_batch_sample(systems, inner: int = 2):
    """The CPU oracle as it stands (unblocked LU with partial pivoting in the
    inner precision, exact residual, refinement to 2^-200) on whole systems,
    all host cores: (systems solved to 2^-200, seconds, threads)."""
    import oracle
    # every core the process may run on (torchrun sets OMP_NUM_THREADS=1 for
    # its ranks, which would leave rank 0's oracle on one core)
    threads = oracle.set_threads(len(os.sched_getaffinity(0)))
    met = 0
    t0 = time.perf_counter()
    for A, b in systems:
        st, x, corr, nres, info = oracle.refine(A, b, inner, target_bits=TARGET_BITS)
        met += int(st == 0 and batch_target_met(x.reshape(-1), [A.shape[1]])[0])
    return met, time.perf_counter() - t0, threads


def cpu_baseline_line(systems, sample_desc):
    met, secs, threads = oracle_batch_sample(systems)
    return {"value": met / secs, "unit": "solves/s", "cores": threads, "kind": "oracle",
            "sample": (f"{sample_desc}: {len(systems)} whole systems, each factored (DD, unblocked), "
                       f"solved and refined to 2^-200 by the oracle; {met} met the target in {secs:.1f} s"),
            "seconds": secs}


def run_reference(args, world, rank):
    """The oracle as it stands on the host cores: the headline metric and
    workload, each step a stratified sample of whole systems of the batch."""
    if rank != 0:
        return 0
    from paper_2107_12550_gb300 import workloads as W
    import oracle
    oracle.build()
    n_list, kap = W.mixed_batch_spec(args.count, N_LO, N_HI, LOG10_KAPPA_LO, LOG10_KAPPA_HI, seed=0)
    ids = stratified_sample(n_list, 32)
    sub_n = [n_list[s] for s in ids]
    A_np, b_np = W.svd_batch(sub_n, [kap[s] for s in ids], seed=0, a_words=A_WORDS, b_words=X_WORDS,
                             processes=len(os.sched_getaffinity(0)), system_ids=ids)
    systems = [batch_system(A_np, b_np, sub_n, i) for i in range(len(ids))]
    vals, secs = [], []
    met = threads = 0
    for it in range(args.warmup + args.steps):
        met, t, threads = oracle_batch_sample(systems)
        if it >= args.warmup:
            vals.append(met / t)
            secs.append(t)
    v = statistics.mean(vals)
    desc = (f"every 32nd system of the {args.count}-system batch in order of n ({len(ids)} whole systems "
            f"per step, DD inner LU, refined to 2^-200; {met} of {len(ids)} met the target)")
    line = {"impl": "reference", "metric": "solves/s at 2^-200 rel. error", "value": v,
            "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(secs) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.count), "systems": args.count, "n_range": [N_LO, N_HI],
                       "log10_kappa_range": [LOG10_KAPPA_LO, LOG10_KAPPA_HI], "global_batch": args.count,
                       "seq_len": 0, "parallelism": "cpu-oracle", "inner": "dd", "target_bits": TARGET_BITS,
                       "l2": "inputs_larger_than_l2"},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": threads, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _time(fn, reps, stream):
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = None
    for _ in range(reps):
        out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def serial_profile(fn, reps):
    """Per-phase library profile of `reps` calls of fn, run with the serial
    schedule (MW_TUNE_LOOKAHEAD 0 for every precision: bitwise the same
    results).  Under the look-ahead a panel runs beside the trailing update,
    so each phase's events would also hold the other's time; wall-clock
    numbers are taken apart, with the look-ahead on."""
    import torch
    from paper_2107_12550_gb300 import _lib as L
    lib = L.lib()
    prev = {w: lib.mw_set_tuning(L.MW_TUNE_LOOKAHEAD, w, 0) for w in (2, 3, 4)}
    try:
        torch.cuda.synchronize()
        L.profile_read(reset=True)
        L.profile_enable(True)
        out = None
        for _ in range(reps):
            out = fn()
        torch.cuda.synchronize()
        L.profile_enable(False)
        return L.profile_read(reset=True), out
    finally:
        for w, v in prev.items():
            lib.mw_set_tuning(L.MW_TUNE_LOOKAHEAD, w, v)


def single_system_td(peak_fp64, steps, sm_max_mhz):
    """The plain FP64-core form on one system: n = 2048, kappa ~ 1e10, QD
    stored, TD LU with the plain trailing update, refined to 2^-200; with the
    FP64-pipe roofline of its dominant kernel k_gemm_plain<TD>."""
    import torch
    from paper_2107_12550_gb300 import _lib as L
    from paper_2107_12550_gb300 import api
    from paper_2107_12550_gb300 import workloads as W
    s = W.svd_system(N, LOG10_KAPPA, seed=0)
    A = torch.from_numpy(s.A).cuda()
    b = torch.from_numpy(s.b).cuda()
    x = torch.empty((X_WORDS, N), dtype=torch.float64, device="cuda")
    work = api.workspace(L.MW_OP_REFINE, INNER, 0, N)
    stream = torch.cuda.current_stream()
    knobs = tuned(INNER, N, "lu")
    f = lambda: api.refine(A, b, INNER, TARGET_BITS, x_words=X_WORDS, work=work, out=x)
    r = f()
    ms, r = _time(f, steps, stream)
    ok = r.converged and exact_ok(x.cpu().numpy(), N)
    prof, _ = serial_profile(f, steps)
    gemm_ms, gemm_launches = prof["gemm_plain"]
    instr = panel_sum_sq(N) * FP64_PER_MSUB_INT[INNER] * steps
    achieved = instr / (gemm_ms * 1e-3) if gemm_ms > 0 else 0.0
    ceiling = FP64_LANES_PER_CLK * sm_max_mhz * 1e6 if sm_max_mhz else None
    lu_ms = sum(prof[p][0] for p in ("panel", "laswp", "trsm", "gemm_plain")) / steps
    out = {"workload": "svd_kappa1e10_n2048_qd_stored_td_inner_plain_refine_to_2^-200", "tuning": knobs,
           "solves_per_s": (1.0 if ok else 0.0) / (ms * 1e-3), "ms_per_solve": ms,
           "corrections": r.corrections, "residuals": r.residuals, "target_met": ok,
           "lu_ms": lu_ms, "lu_td_gops": (2.0 / 3.0) * N ** 3 / (lu_ms * 1e-3) / 1e9 if lu_ms else None,
           "phase_ms_per_solve": {k: v[0] / steps for k, v in prof.items() if v[1]},
           "roofline": {"bound": "alu", "pipe": "fp64", "kernel": "k_gemm_plain<TD>",
                        "achieved": achieved / 1e12, "peak": peak_fp64 / 1e12, "unit": "T FP64 instr/s",
                        "frac": achieved / peak_fp64, "peak_source": "measured: mw_peak_fp64 in this run",
                        "frac_of_fp64_issue_ceiling": achieved / ceiling if ceiling else None,
                        "traffic": GEMM_TD_TRAFFIC_PER_LAUNCH, "traffic_unit": "bytes per launch (ncu)",
                        "algorithmic_per_launch": instr / max(gemm_launches, 1)}}
    # the split-precision DD inner LU on the same system
    reset_knobs()
    work2 = api.workspace(L.MW_OP_REFINE, 2, 1, N)
    g = lambda: api.refine(A, b, 2, TARGET_BITS, update="split", x_words=X_WORDS, work=work2, out=x)
    r2 = g()
    ms2, r2 = _time(g, max(steps, 3), stream)
    ok2 = r2.converged and exact_ok(x.cpu().numpy(), N)
    out["split_dd_inner"] = {"solves_per_s": (1.0 if ok2 else 0.0) / (ms2 * 1e-3), "ms_per_solve": ms2,
                             "corrections": r2.corrections, "target_met": ok2}
    del A, b, x, work, work2
    torch.cuda.empty_cache()
    return out


def batch_comparators(A, b, A_np, b_np, n_list, peak_fp64, sm_max_mhz):
    """The same headline batch through the plain FP64-core DD LU (blocked
    batched, plain multiword GEMM) with the same refinement, and the plain
    batched QD direct LU + solve (no refinement) on every 16th system in
    order of n."""
    import numpy as np
    import torch
    from paper_2107_12550_gb300 import _lib as L
    from paper_2107_12550_gb300 import api
    stream = torch.cuda.current_stream()
    out = {}
    total_n = int(sum(n_list))
    ops = sum((2.0 / 3.0) * m ** 3 for m in n_list)
    x = torch.empty(X_WORDS * total_n, dtype=torch.float64, device="cuda")
    work = api.batch_blocked_workspace(L.MW_OP_REFINE, 2, "plain", n_list)
    f = lambda: api.refine_batched_blocked(A, A_WORDS, b, X_WORDS, n_list, 2, "plain", TARGET_BITS, work=work, out=x)
    f()
    ms, (_, stats) = _time(f, 1, stream)
    met = batch_target_met(x.cpu().numpy(), n_list)
    prof, _ = serial_profile(f, 1)
    lu_ms = sum(prof[p][0] for p in ("panel", "laswp", "trsm", "gemm_plain"))
    pm, tm = blocked_batch_msubs(n_list)
    ph = {k: v[0] for k, v in prof.items() if v[1]}
    out["plain_dd_batched_refine"] = {
        "ms_per_batch": ms, "systems_met": int(sum(met)), "solves_per_s": int(sum(met)) / (ms * 1e-3),
        "lu_ms": lu_ms, "lu_dd_gops": ops / (lu_ms * 1e-3) / 1e9 if lu_ms else None, "phase_ms": ph,
        "panel_fp64_frac_msub_only": pm * FP64_PER_MSUB_INT[2] / (ph["panel"] * 1e-3) / peak_fp64 if ph.get("panel") else None,
        "trsm_fp64_frac_msub_only": tm * FP64_PER_MSUB_INT[2] / (ph["trsm"] * 1e-3) / peak_fp64 if ph.get("trsm") else None}
    del work, x
    sample = stratified_sample(n_list, 16)
    sn = [n_list[s] for s in sample]
    moff, voff = api.batch_offsets(n_list)
    As = np.concatenate([A_np[A_WORDS * moff[s]: A_WORDS * moff[s + 1]] for s in sample])
    bs = np.concatenate([b_np[X_WORDS * voff[s]: X_WORDS * voff[s] + 4 * n_list[s]] for s in sample])
    Asd = torch.from_numpy(As).cuda()
    bsd = torch.from_numpy(bs).cuda()
    wk = api.batch_blocked_workspace(L.MW_OP_LUDECOMP, 4, "plain", sn)
    wks = api.batch_workspace(L.MW_OP_SOLVE, 4, sn)
    LUq = torch.empty_like(Asd)

    def qd_direct():
        LUq.copy_(Asd)
        LU_, piv_, _ = api.ludecomp_batched_blocked(LUq, sn, 4, "plain", work=wk, inplace=True)
        return api.solve_batched(LU_, piv_, bsd, sn, 4, work=wks)

    qd_direct()
    tq, xq = _time(qd_direct, 1, stream)
    xq = xq.cpu().numpy()
    worst = []
    off = 0
    for m in sn:
        Xm = xq[off: off + 4 * m].reshape(4, m)
        off += 4 * m
        worst.append(max(abs(math.fsum([Xm[0, i] - 1.0] + [Xm[c, i] for c in range(1, 4)])) for i in range(m)))
    sample_ops = sum((2.0 / 3.0) * m ** 3 for m in sn)
    out["plain_qd_direct_sample"] = {
        "systems": len(sample), "sample": "every 16th system in order of n", "ms": tq,
        "ms_scaled_to_batch": tq * ops / sample_ops,
        "systems_met": int(sum(1 for e in worst if e <= 2.0 ** -TARGET_BITS)),
        "median_log2_max_error": float(np.median([math.log2(e) if e > 0 else -1100 for e in worst]))}
    del Asd, bsd, LUq
    torch.cuda.empty_cache()
    return out


def extras(steps, peak_fp64, peaks):
    """Comparison measurements beside the headline (same GPU, same run): the
    large DD LU (n = 4096 plain vs split, n = 8192 split), the standalone
    block products (plain vs split, classical vs Strassen) and the
    4096-system batches (n in [16, 256], DD and TD)."""
    import numpy as np
    import torch
    from paper_2107_12550_gb300 import _lib as L
    from paper_2107_12550_gb300 import api
    from paper_2107_12550_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    out = {}
    # large DD LU, n = 4096, plain vs split (LU DD-Gop/s = (2/3) n^3 / t)
    n3 = 4096
    Au = torch.from_numpy(W.uniform_matrix(n3, 2, seed=0)).cuda()
    lu = {}
    knobs3 = {}
    for upd, reps in (("plain", 1), ("split", 3)):
        if upd == "split":
            knobs3 = tuned(2, n3, "split_lu")
        else:
            reset_knobs()
        wk = api.workspace(L.MW_OP_LUDECOMP, 2, 1 if upd == "split" else 0, n3)
        g = lambda: api.ludecomp(Au, 2, upd, work=wk)
        g()
        t, _ = _time(g, reps, stream)
        prof, _ = serial_profile(g, reps)
        lu[upd] = {"ms": t, "dd_gops": (2.0 / 3.0) * n3 ** 3 / (t * 1e-3) / 1e9,
                   "phase_ms": {k: v[0] / reps for k, v in prof.items() if v[1]}}
    # tensor-pipe roofline of the split GEMM: bf16 MMA flops issued per LU
    mma_flops = 0
    for k0 in range(0, n3, 64):
        r0 = k0 + 64
        if r0 >= n3:
            break
        m_t = -(-(n3 - r0) // 128)
        n_t = -(-(n3 - r0) // 16)
        mma_flops += m_t * n_t * 120 * 2 * 128 * 16 * 64
    split_gemm_ms = lu["split"]["phase_ms"].get("gemm_split", 0.0)
    out["lu_dd_n4096"] = {
        "plain_dd_gops": lu["plain"]["dd_gops"], "split_dd_gops": lu["split"]["dd_gops"],
        "plain_ms": lu["plain"]["ms"], "split_ms": lu["split"]["ms"], "split_tuning": knobs3,
        "split_phase_ms": lu["split"]["phase_ms"],
        "split_gemm_roofline": {"bound": "tensor", "kernel": "k_split_gemm (bf16 tcgen05, TMEM)",
                                "achieved": mma_flops / (split_gemm_ms * 1e-3) / 1e12 if split_gemm_ms else None,
                                "peak": peaks.get("bf16_tflops_sustained"), "unit": "TFLOP/s",
                                "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (cuBLAS bf16 GEMM, sustained)",
                                "note": "MMA flops over the kernel time including its exact-recombination epilogue"},
        "plain_gemm_fp64_frac": None,
    }
    pg = lu["plain"]["phase_ms"].get("gemm_plain", 0.0)
    if pg:
        instr = panel_sum_sq(n3) * FP64_PER_MSUB_INT[2]
        out["lu_dd_n4096"]["plain_gemm_fp64_frac"] = instr / (pg * 1e-3) / peak_fp64
    del Au
    # large DD LU, n = 8192, split update (the plain update would take ~11 s)
    n8 = 8192
    A8 = torch.from_numpy(W.uniform_matrix(n8, 2, seed=0)).cuda()
    knobs8 = tuned(2, n8, "split_lu")
    wk8 = api.workspace(L.MW_OP_LUDECOMP, 2, 1, n8)
    g8 = lambda: api.ludecomp(A8, 2, "split", work=wk8)
    g8()
    t8, (_, _, info8) = _time(g8, 1, stream)
    prof8, _ = serial_profile(g8, 1)
    reset_knobs()
    out["lu_dd_n8192_split"] = {"ms": t8, "dd_gops": (2.0 / 3.0) * n8 ** 3 / (t8 * 1e-3) / 1e9, "tuning": knobs8,
                                "info": int(info8.item()),
                                "phase_ms": {k: v[0] for k, v in prof8.items() if v[1]}}
    del A8, wk8
    torch.cuda.empty_cache()
    # the standalone block matrix product C = A B, DD, 4096 x 4096 x 1024,
    # plain vs split (DD-Gop/s = 2 m N K / t: a multiword multiply and an
    # addition per term)
    mg, kg = 4096, 1024
    rg = np.random.default_rng(5)
    ga = np.zeros((2, kg, mg))
    ga[0] = rg.uniform(-1, 1, (kg, mg))
    ga[1] = ga[0] * np.ldexp(rg.uniform(-1, 1, (kg, mg)), -53)
    gb = np.zeros((2, mg, kg))
    gb[0] = rg.uniform(-1, 1, (mg, kg))
    gb[1] = gb[0] * np.ldexp(rg.uniform(-1, 1, (mg, kg)), -53)
    gA = torch.from_numpy(ga).cuda()
    gB = torch.from_numpy(gb).cuda()
    gC = torch.empty((2, mg, mg), dtype=torch.float64, device="cuda")
    del ga, gb
    gm = {}
    for upd, reps in (("plain", 1), ("split", 3)):
        wkg = api.workspace(L.MW_OP_GEMM, 2, 1 if upd == "split" else 0, mg)

        def gstep():
            gC.zero_()
            return api.gemm_add(gC, gA, gB, mg, 2, upd, work=wkg)
        gstep()
        t, _ = _time(gstep, reps, stream)
        gm[upd] = t
    tiles = -(-mg // 128) * -(-mg // 16)
    mma = tiles * (kg // 64) * 120 * 2 * 128 * 16 * 64
    out["gemm_dd_4096x4096x1024"] = {
        "plain_ms": gm["plain"], "split_ms": gm["split"],
        "plain_dd_gops": 2.0 * mg * mg * kg / (gm["plain"] * 1e-3) / 1e9,
        "split_dd_gops": 2.0 * mg * mg * kg / (gm["split"] * 1e-3) / 1e9,
        "split_mma_tflops": mma / (gm["split"] * 1e-3) / 1e12,
        "workload": "C = A B from a zero C (mw_gemm_add), DD entries uniform in [-1, 1]"}
    del gA, gB, gC
    torch.cuda.empty_cache()
    # Strassen's recursion over the block product, DD: plain at n = 2048
    # (levels 0-2), split at n = 4096 (levels 0-1); DD-Gop/s counts the
    # classical 2 n^3 operations
    st = {}
    for upd, ns, lv_list, reps in (("plain", 2048, (0, 1, 2), 1), ("split", 4096, (0, 1), 3)):
        rs = np.random.default_rng(9)
        sa = np.zeros((2, ns, ns))
        sa[0] = rs.uniform(-1, 1, (ns, ns))
        sa[1] = sa[0] * np.ldexp(rs.uniform(-1, 1, (ns, ns)), -53)
        sA = torch.from_numpy(sa).cuda()
        sB = torch.from_numpy(sa[:, ::-1, :].copy()).cuda()
        del sa
        sC = torch.empty_like(sA)
        for lv in lv_list:
            g = lambda: api.gemm_strassen(sA, sB, 2, upd, lv, out=sC)
            g()
            t, _ = _time(g, reps, stream)
            st[f"{upd}_n{ns}_levels{lv}"] = {"ms": t, "dd_gops": 2.0 * ns ** 3 / (t * 1e-3) / 1e9}
        del sA, sB, sC
        torch.cuda.empty_cache()
    out["gemm_strassen_dd"] = st
    # batches of 4096 TD and DD systems, n in [16, 256], one RHS (x_true = ones)
    n_list = [int(v) for v in W.batch_sizes(4096, 16, 256, seed=0)]
    mats = [W.uniform_matrix(m, 3, seed=W.system_seed(0, s), lda=m) for s, m in enumerate(n_list)]
    At = torch.from_numpy(api.pack_matrices(mats, 3)).cuda()
    del mats
    vt = np.zeros(3 * int(sum(n_list)))
    _, voff = api.batch_offsets(n_list)
    for s, m in enumerate(n_list):
        vt[3 * voff[s]: 3 * voff[s] + m] = 1.0
    bt = torch.from_numpy(vt).cuda()
    wkt = api.batch_workspace(L.MW_OP_LUDECOMP, 3, n_list)
    LUt = torch.empty_like(At)

    def batch_step_td():
        LUt.copy_(At)
        LU_, piv_, info_ = api.ludecomp_batched(LUt, n_list, 3, work=wkt, inplace=True)
        return api.solve_batched(LU_, piv_, bt, n_list, 3, work=wkt)

    batch_step_td()
    ttd, _ = _time(batch_step_td, 2, stream)
    ops_td = sum((2.0 / 3.0) * m ** 3 for m in n_list)
    out["batch_4096_td_n16_256"] = {
        "systems": 4096, "n_range": [16, 256], "ms_per_batch": ttd, "systems_per_s": 4096 / (ttd * 1e-3),
        "lu_td_gops": ops_td / (ttd * 1e-3) / 1e9,
        "workload": "uniform TD systems, LU + solve; persistent one-CTA-per-system LU"}
    del At, LUt, bt
    torch.cuda.empty_cache()
    mats = [W.uniform_matrix(m, 2, seed=W.system_seed(0, s), lda=m) for s, m in enumerate(n_list)]
    Ab = torch.from_numpy(api.pack_matrices(mats, 2)).cuda()
    del mats
    vb = np.zeros(2 * int(sum(n_list)))
    _, voff = api.batch_offsets(n_list)
    for s, m in enumerate(n_list):
        vb[2 * voff[s]: 2 * voff[s] + m] = 1.0
    bb = torch.from_numpy(vb).cuda()
    wk = api.batch_workspace(L.MW_OP_LUDECOMP, 2, n_list)
    LUb = torch.empty_like(Ab)
    pivb = torch.empty(int(sum(n_list)), dtype=torch.int64, device="cuda")

    def batch_step():
        LUb.copy_(Ab)
        LU_, piv_, info_ = api.ludecomp_batched(LUb, n_list, 2, work=wk, inplace=True)
        return api.solve_batched(LU_, piv_, bb, n_list, 2, work=wk)

    batch_step()
    tb, _ = _time(batch_step, 2, stream)
    wkb = api.batch_blocked_workspace(L.MW_OP_LUDECOMP, 2, "plain", n_list)

    def batch_step_blocked():
        LUb.copy_(Ab)
        LU_, piv_, info_ = api.ludecomp_batched_blocked(LUb, n_list, 2, "plain", work=wkb, inplace=True)
        return api.solve_batched(LU_, piv_, bb, n_list, 2, work=wk)

    batch_step_blocked()
    tbb, _ = _time(batch_step_blocked, 2, stream)
    ops = sum((2.0 / 3.0) * m ** 3 for m in n_list)
    out["batch_4096_dd_n16_256"] = {
        "systems": 4096, "n_range": [16, 256], "ms_per_batch": tb, "systems_per_s": 4096 / (tb * 1e-3),
        "lu_dd_gops": ops / (tb * 1e-3) / 1e9, "blocked_plain_ms_per_batch": tbb,
        "workload": "uniform DD systems, LU + solve; persistent one-CTA-per-system LU, and the blocked batched LU"}
    del Ab, LUb, bb
    torch.cuda.empty_cache()
    return out


def batch_target_met(x_flat, n_list, words=X_WORDS):
    """Per system: |x_i - 1| <= 2^-200 for every i (math.fsum of the words,
    exact Fraction check near the threshold)."""
    import numpy as np
    lim = 2.0 ** -TARGET_BITS
    met = []
    off = 0
    for n in n_list:
        X = np.asarray(x_flat[off: off + words * n]).reshape(words, n)
        off += words * n
        ok = True
        for i in range(n):
            d = math.fsum([X[0, i] - 1.0] + [X[c, i] for c in range(1, words)])
            if abs(d) > 2.0 * lim:
                ok = False
                break
            if abs(d) >= 0.5 * lim:
                v = sum((Fraction(float(X[c, i])) for c in range(words)), Fraction(0))
                if abs(v - 1) > Fraction(1, 2 ** TARGET_BITS):
                    ok = False
                    break
        met.append(ok)
    return met


def blocked_batch_msubs(n_list, nb=64):
    """Multiword multiply-subtract steps of the blocked batched LU outside the
    trailing update: (panel, TRSM) summed over systems and panel steps."""
    panel = trsm = 0
    for n in n_list:
        for k0 in range(0, n, nb):
            kb = min(nb, n - k0)
            for kk in range(kb):
                panel += (n - k0 - kk - 1) * (kb - kk - 1)
            trsm += max(0, n - k0 - kb) * kb * (kb - 1) // 2
    return panel, trsm


def split_panel_fp64_msubs(n_list, nb: int = 64, leaf: int = 8) -> int:
    """Multiword multiply-subtracts of the split batched panel that run on
    the FP64 pipe: each 8-column leaf's in-panel updates over the rows below
    it, and for every halving (64 -> 32 -> 16 -> 8) the right half's top h
    rows solved with the left half's unit lower triangle (h^2 (h - 1) / 2)."""
    tot = 0
    for n in n_list:
        for k0 in range(0, n, nb):
            for c in range(0, min(nb, n - k0), leaf):
                w = min(leaf, n - k0 - c)
                rows = n - k0 - c
                tot += sum((rows - kk - 1) * (w - kk - 1) for kk in range(w))
            h = nb // 2
            while h >= leaf:
                for c_off in range(0, nb, 2 * h):
                    if n - k0 - c_off - h > 0:
                        hh = min(h, n - k0 - c_off - h)
                        tot += hh * h * (h - 1) // 2
                h //= 2
    return tot


def headline_rooflines(prof, reps, n_list, stats, peak_fp64, peaks, sm_max_mhz):
    """Per-kernel rooflines of the headline step from one profiled pass
    (reps calls): the batched substitution and the panel phase against the
    FP64 pipe, the trailing split update against the bf16 tensor pipe, the
    exact residual in exact products per second.  Work per unit:
    substitution n^2 multiword multiply-subtracts per solve (FP64_PER_MSUB_INT
    FP64 instructions each); split update SPLIT_TILE_FLOPS bf16 flops per
    128 x 16 tile; residual n^2 * 4 * 8 word products per evaluation."""
    ceiling = FP64_LANES_PER_CLK * sm_max_mhz * 1e6 if sm_max_mhz else None
    out = []
    solves = sum((1 + int(stats[s, 0])) * n_list[s] ** 2 for s in range(len(n_list)))
    t = prof["batch_solve"][0] / reps
    if t > 0:
        a = solves * FP64_PER_MSUB_INT[2] / (t * 1e-3)
        out.append({"kernel": "k_solve_batched<DD>", "ms": t, "bound": "alu", "pipe": "fp64",
                    "achieved": a / 1e12, "peak": peak_fp64 / 1e12, "unit": "T FP64 instr/s",
                    "frac": a / peak_fp64, "peak_source": "measured: mw_peak_fp64 in this run",
                    "frac_of_fp64_issue_ceiling": a / ceiling if ceiling else None,
                    "traffic": (SOLVE_BATCHED_TRAFFIC_PER_MSUB * solves / max(prof["batch_solve"][1] / reps, 1)
                                if SOLVE_BATCHED_TRAFFIC_PER_MSUB else None),
                    "algorithmic_per_launch": solves * FP64_PER_MSUB_INT[2] / max(prof["batch_solve"][1] / reps, 1),
                    "unit_of_work": "n^2 DD multiply-subtracts per system and solve"})
    t = prof["gemm_split"][0] / reps
    if t > 0:
        fl = split_trail_mma_flops(n_list)
        pk = peaks.get("bf16_tflops_sustained")
        a = fl / (t * 1e-3) / 1e12
        out.append({"kernel": "k_bsplit_gemm (trailing updates)", "ms": t, "bound": "tensor",
                    "achieved": a, "peak": pk, "unit": "TFLOP/s", "frac": a / pk if pk else None,
                    "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained",
                    "unit_of_work": "120 bf16 digit-pair MMAs of 128 x 16 x 64 per output tile",
                    "traffic": None})
    t = prof["panel"][0] / reps
    if t > 0:
        pm = split_panel_fp64_msubs(n_list)
        a = pm * FP64_PER_MSUB_INT[2] / (t * 1e-3)
        out.append({"kernel": "panel phase on the FP64 pipe (k_bpanel 8-column leaves, k_btrsm_sub)", "ms": t,
                    "bound": "alu", "pipe": "fp64", "achieved": a / 1e12, "peak": peak_fp64 / 1e12,
                    "unit": "T FP64 instr/s", "frac": a / peak_fp64,
                    "peak_source": "measured: mw_peak_fp64 in this run",
                    "unit_of_work": "the leaves' in-panel multiply-subtracts and the right halves' unit "
                                    "lower solves (the inner products run on the tensor cores, timed apart)",
                    "traffic": None})
    t = prof["residual"][0] / reps
    if t > 0:
        prods = sum(int(stats[s, 1]) * n_list[s] ** 2 * A_WORDS * X_WORDS for s in range(len(n_list)))
        out.append({"kernel": "k_bt_residual", "ms": t, "bound": "alu", "achieved": prods / (t * 1e-3) / 1e12,
                    "peak": None, "unit": "T exact word products/s", "frac": None,
                    "unit_of_work": "n^2 x 4 x 8 exact word products per evaluation", "traffic": None})
    return out


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        return run_reference(args, world, rank)

    import numpy as np
    import torch
    from paper_2107_12550_gb300 import _lib as L
    from paper_2107_12550_gb300 import api
    from paper_2107_12550_gb300 import build as B
    from paper_2107_12550_gb300 import workloads as W

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    peaks = measured_peaks()
    n_list, kap = W.mixed_batch_spec(args.count, N_LO, N_HI, LOG10_KAPPA_LO, LOG10_KAPPA_HI, seed=rank)
    t0 = time.time()
    procs = max(1, len(os.sched_getaffinity(0)) // world)
    A_np, b_np = W.svd_batch(n_list, kap, seed=rank, a_words=A_WORDS, b_words=X_WORDS, processes=procs)
    gen_s = time.time() - t0
    A = torch.from_numpy(A_np).cuda()
    b = torch.from_numpy(b_np).cuda()
    total_n = int(sum(n_list))
    x = torch.empty(X_WORDS * total_n, dtype=torch.float64, device="cuda")
    work = api.batch_blocked_workspace(L.MW_OP_REFINE, 2, "split", n_list)
    stream = torch.cuda.current_stream()

    def step():
        return api.refine_batched_blocked(A, A_WORDS, b, X_WORDS, n_list, 2, "split", TARGET_BITS,
                                          work=work, out=x)

    peak_fp64 = api.peak_fp64()            # project microbenchmark, instructions/s
    knobs = tuned(2, N_HI, "batched_split")
    for _ in range(max(args.warmup, 1)):
        _, stats = step()
    torch.cuda.synchronize()
    met_ref = batch_target_met(x.cpu().numpy(), n_list)

    # the whole step captured once as a CUDA graph (the blocked batched LU and
    # the refinement loop as a while node whose condition the device sets);
    # the timed region replays it.  Replays must reproduce the eager step.
    api.batch_plan_cache(True)
    st_buf = torch.empty((args.count, 4), dtype=torch.int64, device="cuda")

    def step_into():
        _, s_ = step()
        st_buf.copy_(s_)

    step_into()
    torch.cuda.synchronize()
    x_eager, st_eager = x.clone(), st_buf.clone()
    side = torch.cuda.Stream()
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        step_into()
    stream.wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step_into()
    x.zero_()
    graph.replay()
    torch.cuda.synchronize()
    graph_bitwise = bool(torch.equal(x, x_eager) and torch.equal(st_buf, st_eager))
    # eager steps timed apart, for comparison
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for _ in range(max(2, args.steps // 2)):
        step()
    g1.record(stream)
    torch.cuda.synchronize()
    eager_ms = g0.elapsed_time(g1) / max(2, args.steps // 2)

    # ---- timed region: K steps, device-resident inputs -------------------
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    met = batch_target_met(x.cpu().numpy(), n_list)
    st = st_buf.cpu().numpy()
    met_per_step = int(sum(met)) if met == met_ref else min(int(sum(met)), int(sum(met_ref)))
    t_max, solved = combine_ranks(ms, args.steps * met_per_step, "cuda")
    value = solved / (t_max * 1e-3)

    # ---- one profiled pass (not timed above): phases and kernel rooflines -
    # Run with the serial schedule (MW_TUNE_LOOKAHEAD 0: bitwise the same
    # results), so that no phase's events overlap another's and each phase
    # time is its kernels' own duration.
    prof, (_, pst) = serial_profile(step, 1)
    sm_max = clk.get("sm_max_mhz") or peaks.get("sm_max_mhz")
    roofs = headline_rooflines(prof, 1, n_list, pst.cpu().numpy(), peak_fp64, peaks, sm_max)
    dominant = max(roofs, key=lambda r: r["ms"]) if roofs else None
    launches = sum(c for _, c in prof.values())
    ops = sum((2.0 / 3.0) * m ** 3 for m in n_list)
    lu_ms = sum(prof[p][0] for p in ("panel", "laswp", "trsm", "gemm_plain", "gemm_split", "split_aux", "panel_inner"))

    # ---- end to end through the public API with host buffers -------------
    # Every step copies its inputs (A, b) from pinned host memory and reads x
    # and the per-system statistics back.  Two schedules are timed and the
    # faster is reported (both are recorded): "sequential", each step's copy,
    # graph replay and read-back in order on one stream; "overlapped", two
    # input buffers, each with its own captured graph, so that step k+1's
    # host-to-device copy runs on a copy stream while step k computes (the
    # copy into a buffer waits until the step that last read it finished).
    A_h = torch.from_numpy(A_np).pin_memory()
    b_h = torch.from_numpy(b_np).pin_memory()
    A2, b2 = torch.empty_like(A), torch.empty_like(b)
    A2.copy_(A)
    b2.copy_(b)
    x2, st2 = torch.empty_like(x), torch.empty_like(st_buf)

    def step_into2():
        _, s_ = api.refine_batched_blocked(A2, A_WORDS, b2, X_WORDS, n_list, 2, "split", TARGET_BITS,
                                           work=work, out=x2)
        st2.copy_(s_)

    step_into2()
    torch.cuda.synchronize()
    graph2 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph2):
        step_into2()
    bufs = [(A, b, x, st_buf, graph), (A2, b2, x2, st2, graph2)]
    x_h = [torch.empty_like(x, device="cpu").pin_memory() for _ in range(2)]
    s_h = [torch.empty((args.count, 4), dtype=torch.int64).pin_memory() for _ in range(2)]
    # each step's inputs go over in N_COPY chunks on as many copy streams, so
    # that several copy engines share the host-to-device transfer
    N_COPY = 8
    copy_streams = [torch.cuda.Stream() for _ in range(N_COPY)]
    ev_in = [[torch.cuda.Event() for _ in range(N_COPY)] for _ in range(2)]
    ev_used = [torch.cuda.Event(), torch.cuda.Event()]
    e2e_steps = max(4, args.steps // 2)
    A_hf, b_hf = A_h.reshape(-1), b_h.reshape(-1)
    cut = [A_hf.numel() * c // N_COPY for c in range(N_COPY + 1)]

    def load(k, after=None):
        """Copy step k's inputs into buffer k % 2; ev_in[k % 2] marks them done."""
        i = k % 2
        Af = bufs[i][0].reshape(-1)
        for c, cs in enumerate(copy_streams):
            with torch.cuda.stream(cs):
                if after is not None:
                    cs.wait_event(after)
                if k >= 2:
                    cs.wait_event(ev_used[i])
                Af[cut[c]:cut[c + 1]].copy_(A_hf[cut[c]:cut[c + 1]], non_blocking=True)
                if c == 0:
                    bufs[i][1].reshape(-1).copy_(b_hf, non_blocking=True)
                ev_in[i][c].record(cs)

    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    load(0, after=f0)
    for k in range(e2e_steps):
        i = k % 2
        if k + 1 < e2e_steps:
            load(k + 1)
        for ev in ev_in[i]:
            stream.wait_event(ev)
        bufs[i][4].replay()
        ev_used[i].record(stream)
        x_h[i].copy_(bufs[i][2], non_blocking=True)
        s_h[i].copy_(bufs[i][3], non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    ovl_ms = f0.elapsed_time(f1) / e2e_steps
    ovl_met = min(int(sum(batch_target_met(x_h[i].numpy(), n_list))) for i in range(2))
    # sequential schedule on the first buffer set
    torch.cuda.synchronize()
    f0.record(stream)
    for k in range(e2e_steps):
        ev_used[0].record(stream)
        load(0, after=ev_used[0])            # buffer 0, after the previous step
        for ev in ev_in[0]:
            stream.wait_event(ev)
        graph.replay()
        x_h[0].copy_(x, non_blocking=True)
        s_h[0].copy_(st_buf, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    seq_ms = f0.elapsed_time(f1) / e2e_steps
    seq_met = int(sum(batch_target_met(x_h[0].numpy(), n_list)))
    if seq_ms <= ovl_ms:
        e2e_sched, e2e_ms, e2e_met = "sequential", seq_ms, seq_met
    else:
        e2e_sched, e2e_ms, e2e_met = "overlapped", ovl_ms, ovl_met
    # whole job, like `value`: systems met on all ranks over the slowest rank's time
    e2e_t_max, e2e_solved = combine_ranks(e2e_ms, e2e_met, "cuda")
    e2e_val = e2e_solved / (e2e_t_max * 1e-3)
    del A_h, A2, b2, x2, graph2
    # every graph is captured; the comparisons below make eager calls with
    # work buffers of their own, which must not be taken for resident plans
    # (a freed buffer's address can come back for a new one)
    api.batch_plan_cache(False)

    line = {
        "metric": "solves/s at 2^-200 rel. error",
        "value": value,
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(args.count), "systems": args.count, "n_range": [N_LO, N_HI],
                   "log10_kappa_range": [LOG10_KAPPA_LO, LOG10_KAPPA_HI], "global_batch": args.count * world,
                   "seq_len": 0, "parallelism": f"replicas{world}", "inner": "dd", "lu_update": "split",
                   "a_words": A_WORDS, "b_words": X_WORDS, "x_words": X_WORDS, "target_bits": TARGET_BITS,
                   "tuning": {"op": "batched_split", "applied": knobs},
                   "l2": f"inputs_larger_than_l2 (A: {A_np.nbytes / 1e9:.1f} GB QD)"},
        "systems_met_per_step": met_per_step,
        "cuda_graph": {"replay_bitwise_equal_to_eager": graph_bitwise, "eager_ms_per_step": eager_ms},
        "corrections_max": int(st[:, 0].max()), "corrections_mean": float(st[:, 0].mean()),
        "generation_s": gen_s,
        "lu_ms": lu_ms,
        "lu_dd_gops": ops / (lu_ms * 1e-3) / 1e9 if lu_ms > 0 else None,
        "phase_ms_per_step": {k: v[0] for k, v in prof.items() if v[1]},
        "roofline": dominant,
        "rooflines": roofs,
        "gpu_launches": launches * args.steps,
        "clocks": clk,
        "e2e": {"value": e2e_val, "unit": "solves/s", "steps": e2e_steps, "ms_per_step": e2e_t_max,
                "h2d_bytes_per_step": int(A_np.nbytes + b_np.nbytes),
                "d2h_bytes_per_step": int(x.numel() * 8 + args.count * 4 * 8),
                "schedule": e2e_sched,
                "ms_per_step_by_schedule": {"sequential": seq_ms, "overlapped": ovl_ms},
                "copy_streams": N_COPY,
                "schedules": {"sequential": "copy in (chunked over the copy streams), graph replay, read "
                                            "back, each step after the previous one",
                              "overlapped": "two input buffers and graphs: step k+1's host-to-device copy "
                                            "runs on the copy streams during step k"}},
    }
    if rank == 0 and world == 1 and not args.no_extras:
        ex = {"comparators": batch_comparators(A, b, A_np, b_np, n_list, peak_fp64, sm_max)}
        del graph, A, b, x, work
        torch.cuda.empty_cache()
        ex["comparators"]["single_system_plain_td_n2048"] = single_system_td(peak_fp64, 3, sm_max)
        ex.update(extras(args.steps, peak_fp64, peaks))
        r = ex.get("lu_dd_n4096", {}).get("split_gemm_roofline")
        if r and r.get("achieved") and r.get("peak"):
            r["frac"] = r["achieved"] / r["peak"]
        line["extras"] = ex
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ids = stratified_sample(n_list, 8)
        systems = [batch_system(A_np, b_np, n_list, s) for s in ids]
        line["cpu_baseline"] = cpu_baseline_line(
            systems, f"every 8th system of the {args.count}-system batch in order of n")
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
