#!/usr/bin/env python3
"""Benchmark of the multiword direct solver + mixed precision iterative
refinement (Kouya, arXiv 2107.12550, Section 2 Listing 1 and Section 3).

Workload (one GPU): one dense system of order n = 2048, A = U diag(sigma)
V^T with U, V Haar-orthogonal (Householder QR of Gaussian matrices, quantised
to 2^-20), sigma geometric from 1 to 2^-33 (kappa ~ 1e10), stored exactly in
QD (4 words); b = A * ones exactly in 8 words, so x* = ones.  A step is one
call of the library's refinement: TD LU with partial pivoting (plain FP64
trailing update), TD substitution, and the loop r = b - A x (exact, rounded to
8 words = 424 bits), z = solve(2^-e r), x = RN_8(x + 2^e z) until the
correction is below 2^-202 ||x||.  Metric: systems solved to 2^-200 relative
forward error per second, from device-resident (A, b) to device-resident x.

Multi-GPU: every rank solves its own independent system (seeded by rank), no
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

N = 2048
LOG10_KAPPA = 10.0
INNER = 3                 # TD
TARGET_BITS = 200
X_WORDS = 8
WORKLOAD = "svd_kappa1e10_n2048_qd_stored_td_inner_refine_to_2^-200"

# FP64 instructions of one multiword multiply + subtraction (the elimination
# step), counted from the algorithms in csrc/mw_arith.cuh on their typical
# (all error terms non-zero) path
FP64_PER_MSUB = {2: 29, 3: 117, 4: 196}

# DRAM bytes (read + write) per launch of the TD plain trailing update in this
# workload: ncu dram__bytes_read.sum + dram__bytes_write.sum over the 124
# launches of one bench run (warm-up, one step, the end-to-end steps),
# averaged per launch.  Must be re-measured whenever k_gemm_plain changes.
GEMM_TD_TRAFFIC_PER_LAUNCH = 40.40e6

CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="mwlu", choices=["mwlu", "reference"])
    p.add_argument("--n", type=int, default=N)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the split / large-LU / batched comparison measurements")
    p.add_argument("--no-mixed-batch", action="store_true",
                   help="skip the 512-system mixed-precision batched refinement (about a minute of input generation)")
    return p.parse_args()


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


def cpu_oracle_sample(n: int, sys_A, sys_b, corrections: int, residuals: int, m_steps: int = 128):
    """Time the CPU oracle on a bounded sample of the same workload: the
    first m_steps elimination steps of the same n = 2048 TD LU (scaled to the
    full factorisation by the exact multiply-subtract count), plus one full
    oracle solve and one full exact residual (scaled by the step's solve and
    residual counts)."""
    import oracle
    import numpy as np
    threads = oracle.set_threads(0)
    t0 = time.perf_counter()
    LU, piv, info = oracle.lu_steps(INNER, sys_A, m_steps)
    t_lu_sample = time.perf_counter() - t0
    full = sum((n - k - 1) ** 2 for k in range(n))
    part = sum((n - k - 1) ** 2 for k in range(min(m_steps, n)))
    t_lu = t_lu_sample * full / part
    # solve and residual at full size (the solve runs on the partially
    # factored matrix: same operation count; the residual uses an 8-word
    # iterate with every word non-zero, as in the later refinement steps)
    t0 = time.perf_counter()
    oracle.solve(INNER, LU, piv, sys_b)
    t_solve = time.perf_counter() - t0
    g = np.random.default_rng(1)
    x8 = np.stack([np.ldexp(1.0 + g.uniform(-0.5, 0.5, n) * (c > 0), -60 * c) for c in range(X_WORDS)])
    t0 = time.perf_counter()
    oracle.residual(sys_A, sys_b, x8, X_WORDS)
    t_res = time.perf_counter() - t0
    t_total = t_lu + (1 + corrections) * t_solve + residuals * t_res
    sample_s = t_lu_sample + t_solve + t_res
    return {
        "value": 1.0 / t_total,
        "unit": "solves/s",
        "cores": threads,
        "kind": "oracle",
        "sample": (f"first {m_steps} of {n} elimination steps of the same TD LU "
                   f"({t_lu_sample:.1f} s, scaled x{full / part:.2f} by multiply-subtract count), "
                   f"one full TD solve ({t_solve:.2f} s, x{1 + corrections}) and one full exact "
                   f"8-word residual ({t_res:.2f} s, x{residuals}); {sample_s:.1f} s of CPU work"),
        "seconds_per_solve": t_total,
    }


def run_reference(args, world, rank):
    """The oracle as it stands on the host cores, same metric and config."""
    if rank != 0:
        return 0
    from paper_2107_12550_gb300 import workloads as W
    import oracle
    oracle.build()
    s = W.svd_system(args.n, LOG10_KAPPA, seed=0)
    vals = []
    info = None
    for it in range(args.warmup + args.steps):
        info = cpu_oracle_sample(args.n, s.A, s.b, corrections=2, residuals=3,
                                 m_steps=max(8, min(64, args.n)))
        if it >= args.warmup:
            vals.append(info["seconds_per_solve"])
    t = statistics.mean(vals)
    v = 1.0 / t
    line = {"impl": "reference", "metric": "solves/s at 2^-200 rel. error", "value": v,
            "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": args.n, "global_batch": 1, "seq_len": 0,
                       "parallelism": "cpu-oracle", "inner": "td", "target_bits": TARGET_BITS,
                       "l2": "inputs_larger_than_l2"},
            "cpu_baseline": {"value": v, "unit": "solves/s", "cores": info["cores"],
                             "kind": "oracle", "sample": info["sample"]},
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


def extras(A, b, n, steps, peak_fp64):
    """Comparison measurements beside the headline (same GPU, same run):
    the split-precision DD inner solver on the same system, the large DD LU
    (n = 4096) plain vs split, and a 4096-system batch (n in [16, 256])."""
    import numpy as np
    import torch
    from paper_2107_12550_gb300 import _lib as L
    from paper_2107_12550_gb300 import api
    from paper_2107_12550_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    out = {}
    # split DD inner refinement of the same n = 2048 system
    x = torch.empty((X_WORDS, n), dtype=torch.float64, device="cuda")
    work = api.workspace(L.MW_OP_REFINE, 2, 1, n)
    f = lambda: api.refine(A, b, 2, TARGET_BITS, update="split", x_words=X_WORDS, work=work, out=x)
    r = f()
    ms, r = _time(f, max(steps, 3), stream)
    ok = r.converged and exact_ok(x.cpu().numpy(), n)
    out["split_dd_inner_refine"] = {"solves_per_s": (1.0 if ok else 0.0) / (ms * 1e-3), "ms_per_solve": ms,
                                    "corrections": r.corrections, "target_met": ok,
                                    "workload": "same system as the headline, DD inner LU with the split update"}
    # large DD LU, n = 4096, plain vs split (LU DD-Gop/s = (2/3) n^3 / t)
    n3 = 4096
    Au = torch.from_numpy(W.uniform_matrix(n3, 2, seed=0)).cuda()
    lu = {}
    for upd, reps in (("plain", 1), ("split", 3)):
        wk = api.workspace(L.MW_OP_LUDECOMP, 2, 1 if upd == "split" else 0, n3)
        g = lambda: api.ludecomp(Au, 2, upd, work=wk)
        g()
        L.profile_read(reset=True)
        L.profile_enable(True)
        t, _ = _time(g, reps, stream)
        L.profile_enable(False)
        prof = L.profile_read(reset=True)
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
        "plain_ms": lu["plain"]["ms"], "split_ms": lu["split"]["ms"],
        "split_phase_ms": lu["split"]["phase_ms"],
        "split_gemm_roofline": {"bound": "tensor", "kernel": "k_split_gemm (bf16 tcgen05, TMEM)",
                                "achieved": mma_flops / (split_gemm_ms * 1e-3) / 1e12 if split_gemm_ms else None,
                                "peak": None, "unit": "TFLOP/s",
                                "note": "MMA flops over the kernel time including its exact-recombination epilogue"},
        "plain_gemm_fp64_frac": None,
    }
    pg = lu["plain"]["phase_ms"].get("gemm_plain", 0.0)
    if pg:
        instr = panel_sum_sq(n3) * FP64_PER_MSUB[2]
        out["lu_dd_n4096"]["plain_gemm_fp64_frac"] = instr / (pg * 1e-3) / peak_fp64
    del Au
    # large DD LU, n = 8192, split update (the plain update would take ~11 s)
    n8 = 8192
    A8 = torch.from_numpy(W.uniform_matrix(n8, 2, seed=0)).cuda()
    wk8 = api.workspace(L.MW_OP_LUDECOMP, 2, 1, n8)
    g8 = lambda: api.ludecomp(A8, 2, "split", work=wk8)
    g8()
    L.profile_read(reset=True)
    L.profile_enable(True)
    t8, (_, _, info8) = _time(g8, 1, stream)
    L.profile_enable(False)
    prof8 = L.profile_read(reset=True)
    out["lu_dd_n8192_split"] = {"ms": t8, "dd_gops": (2.0 / 3.0) * n8 ** 3 / (t8 * 1e-3) / 1e9,
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


def mixed_batch_refine(peak_fp64, count=512):
    """Batched mixed-precision refinement: `count` SVD systems, n uniform in
    [64, 1024], log10 kappa uniform in [4, 20], A stored in QD, b = A * ones
    exact in 8 words.  Split-update DD inner LU (blocked batched) + exact
    residual + refinement to 2^-200, against the plain FP64-core DD inner LU
    with the same refinement and the plain QD direct LU (a stratified sample
    of the systems, no refinement)."""
    import numpy as np
    import torch
    from paper_2107_12550_gb300 import _lib as L
    from paper_2107_12550_gb300 import api
    from paper_2107_12550_gb300 import workloads as W
    stream = torch.cuda.current_stream()
    n_list, kap = W.mixed_batch_spec(count, 64, 1024, 4.0, 20.0, seed=0)
    t0 = time.time()
    A_np, b_np = W.svd_batch(n_list, kap, seed=0, a_words=4, b_words=X_WORDS,
                             processes=len(os.sched_getaffinity(0)))
    gen_s = time.time() - t0
    A = torch.from_numpy(A_np).cuda()
    b = torch.from_numpy(b_np).cuda()
    total_n = int(sum(n_list))
    ops = sum((2.0 / 3.0) * m ** 3 for m in n_list)
    out = {"systems": count, "n_range": [64, 1024], "log10_kappa_range": [4, 20],
           "generation_s": gen_s, "a_words": 4, "b_words": X_WORDS, "target_bits": TARGET_BITS}
    x = torch.empty(X_WORDS * total_n, dtype=torch.float64, device="cuda")
    for name, upd, reps in (("split_dd_refine", "split", 2), ("plain_dd_refine", "plain", 1)):
        work = api.batch_blocked_workspace(L.MW_OP_REFINE, 2, upd, n_list)
        f = lambda: api.refine_batched_blocked(A, 4, b, X_WORDS, n_list, 2, upd, TARGET_BITS, work=work, out=x)
        f()
        L.profile_read(reset=True)
        L.profile_enable(True)
        ms, (_, stats) = _time(f, reps, stream)
        L.profile_enable(False)
        prof = L.profile_read(reset=True)
        st = stats.cpu().numpy()
        met = batch_target_met(x.cpu().numpy(), n_list)
        lu_ms = sum(prof[p][0] for p in ("panel", "laswp", "trsm", "gemm_plain", "gemm_split", "split_aux")) / reps
        out[name] = {"ms_per_batch": ms, "systems_met": int(sum(met)),
                     "solves_per_s": int(sum(met)) / (ms * 1e-3),
                     "converged": int((st[:, 3] == 0).sum()),
                     "corrections_max": int(st[:, 0].max()), "corrections_mean": float(st[:, 0].mean()),
                     "lu_ms": lu_ms, "lu_dd_gops": ops / (lu_ms * 1e-3) / 1e9 if lu_ms else None,
                     "phase_ms": {k: v[0] / reps for k, v in prof.items() if v[1]},
                     "gpu_launches": int(sum(c for _, c in prof.values()) / reps)}
        del work
    # FP64-pipe fractions of the plain path's panel and TRSM kernels
    # (multiply-subtract instructions only: divisions and compares are not
    # counted).  The split path moves most of that work onto the tensor cores
    # (recursive panel, TRSM through L11^-1), so it has no such fraction.
    pm, tm = blocked_batch_msubs(n_list)
    ph = out["plain_dd_refine"]["phase_ms"]
    for key, cnt in (("panel", pm), ("trsm", tm)):
        t = ph.get(key, 0.0)
        out["plain_dd_refine"][key + "_fp64_frac_msub_only"] = (
            cnt * FP64_PER_MSUB[2] / (t * 1e-3) / peak_fp64 if t else None)
    # plain QD direct LU + solve (no refinement) on every 16th system by order
    order = sorted(range(count), key=lambda s: n_list[s])
    sample = order[::16]
    sn = [n_list[s] for s in sample]
    moff, voff = api.batch_offsets(n_list)
    As = np.concatenate([A_np[4 * moff[s]: 4 * moff[s + 1]] for s in sample])
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
        X = xq[off: off + 4 * m].reshape(4, m)
        off += 4 * m
        worst.append(max(abs(math.fsum([X[0, i] - 1.0] + [X[c, i] for c in range(1, 4)])) for i in range(m)))
    sample_ops = sum((2.0 / 3.0) * m ** 3 for m in sn)
    out["qd_direct_sample"] = {
        "systems": len(sample), "sample": "every 16th system in order of n", "ms": tq,
        "ms_scaled_to_batch": tq * ops / sample_ops,
        "systems_met": int(sum(1 for e in worst if e <= 2.0 ** -TARGET_BITS)),
        "median_log2_max_error": float(np.median([math.log2(e) if e > 0 else -1100 for e in worst]))}
    out["workload"] = ("SVD systems (A = U diag(sigma) V^T exact, QD stored), per-system seeds; "
                       "one call of the blocked batched refinement per batch")
    del A, b, Asd, bsd, LUq, x
    torch.cuda.empty_cache()
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
    n = args.n
    s = W.svd_system(n, LOG10_KAPPA, seed=rank)
    A = torch.from_numpy(s.A).cuda()
    b = torch.from_numpy(s.b).cuda()
    x = torch.empty((X_WORDS, n), dtype=torch.float64, device="cuda")
    work = api.workspace(L.MW_OP_REFINE, INNER, 0, n)
    stream = torch.cuda.current_stream()

    def step():
        return api.refine(A, b, INNER, TARGET_BITS, x_words=X_WORDS, work=work, out=x)

    peak_fp64 = api.peak_fp64()            # project microbenchmark, instructions/s
    res = None
    for _ in range(max(args.warmup, 1)):
        res = step()
    torch.cuda.synchronize()
    ok = res.converged and exact_ok(x.cpu().numpy(), n)
    corrections, residuals = res.corrections, res.residuals

    # ---- timed region: K steps, device-resident inputs -------------------
    L.profile_read(reset=True)
    L.profile_enable(True)
    clocks = ClockSampler(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        res = step()
        ok = ok and res.converged
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    L.profile_enable(False)
    prof = L.profile_read(reset=True)
    ms = e0.elapsed_time(e1)
    ok = ok and exact_ok(x.cpu().numpy(), n)
    t_max, solved = combine_ranks(ms, args.steps * (1 if ok else 0), "cuda")
    value = solved / (t_max * 1e-3)

    # roofline of the dominant kernel: the plain TD trailing update
    gemm_ms, gemm_launches = prof["gemm_plain"]
    msubs_per_lu = panel_sum_sq(n)
    instr = msubs_per_lu * FP64_PER_MSUB[INNER] * args.steps
    achieved = instr / (gemm_ms * 1e-3) / 1e12 if gemm_ms > 0 else 0.0
    peak = peak_fp64 / 1e12
    lu_ms = sum(prof[p][0] for p in ("panel", "laswp", "trsm", "gemm_plain")) / args.steps
    launches = sum(c for _, c in prof.values())

    # ---- end to end through the public API with host buffers -------------
    A_h = torch.from_numpy(s.A).pin_memory()
    b_h = torch.from_numpy(s.b).pin_memory()
    x_h = torch.empty((X_WORDS, n), dtype=torch.float64).pin_memory()
    A_d = torch.empty_like(A)
    b_d = torch.empty_like(b)
    e2e_steps = max(2, args.steps // 2)
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(e2e_steps):
        A_d.copy_(A_h, non_blocking=True)
        b_d.copy_(b_h, non_blocking=True)
        r2 = api.refine(A_d, b_d, INNER, TARGET_BITS, x_words=X_WORDS, work=work, out=x)
        x_h.copy_(x, non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = f0.elapsed_time(f1) / e2e_steps
    e2e_ok = r2.converged and exact_ok(x_h.numpy(), n)
    e2e_val = (1.0 if e2e_ok else 0.0) / (e2e_ms * 1e-3) * world

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
        "config": {"workload": WORKLOAD, "n": n, "global_batch": world, "seq_len": 0,
                   "parallelism": f"replicas{world}", "inner": "td", "lu_update": "plain",
                   "a_words": 4, "b_words": 8, "x_words": X_WORDS, "target_bits": TARGET_BITS,
                   "l2": "inputs_larger_than_l2 (A: 134 MB QD; LU copy 100 MB)"},
        "corrections": corrections,
        "residuals": residuals,
        "lu_ms": lu_ms,
        "lu_td_gops": (2.0 / 3.0) * n ** 3 / (lu_ms * 1e-3) / 1e9 if lu_ms > 0 else None,
        "phase_ms_per_step": {k: v[0] / args.steps for k, v in prof.items() if v[1]},
        "roofline": {"bound": "alu", "pipe": "fp64", "kernel": "k_gemm_plain<TD>",
                     "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "flop": "one FP64 instruction (DADD/DMUL/DFMA)",
                     "peak_source": "measured: mw_peak_fp64 microbenchmark in this run",
                     "frac": achieved / peak if peak else None, "traffic": GEMM_TD_TRAFFIC_PER_LAUNCH,
                     "traffic_unit": "bytes per launch (ncu)",
                     "algorithmic_per_launch": instr / max(gemm_launches, 1)},
        "gpu_launches": launches,
        "clocks": clk,
        "e2e": {"value": e2e_val, "unit": "solves/s",
                "h2d_bytes_per_step": int(s.A.nbytes + s.b.nbytes),
                "d2h_bytes_per_step": int(x.numel() * 8)},
    }
    if rank == 0 and world == 1 and not args.no_extras:
        line["extras"] = extras(A, b, n, args.steps, peak_fp64)
        if not args.no_mixed_batch:
            line["extras"]["mixed_batch_refine_512"] = mixed_batch_refine(peak_fp64)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_oracle_sample(n, s.A, s.b, corrections, residuals)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
