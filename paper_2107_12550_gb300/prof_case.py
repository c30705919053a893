"""Run one library operation on a synthetic case, for profilers.

    python -m paper_2107_12550_gb300.prof_case --op lu --prec 3 --n 4096

Ops: lu (ludecomp), solve, residual, refine, batched_lu (persistent batched
LU), batched_refine (blocked batched LU + refinement of SVD systems with n in
[64, nmax] and kappa log-uniform in [1e4, 1e20]).  Uniform matrices for
lu/solve/residual, the kappa = 1e10 SVD-built matrix for refine.  Exits
non-zero if the library reports an error or a system misses its target.
"""
from __future__ import annotations

import argparse
import sys
import time


def main(argv=None) -> int:
    p = argparse.ArgumentParser()
    p.add_argument("--op", default="lu", choices=["lu", "solve", "residual", "refine", "batched_lu",
                                                   "batched_refine"])
    p.add_argument("--count", type=int, default=512, help="systems in a batch (batched_lu)")
    p.add_argument("--nmax", type=int, default=256, help="largest order in a batch (batched_lu)")
    p.add_argument("--prec", type=int, default=3)
    p.add_argument("--n", type=int, default=2048)
    p.add_argument("--update", default="plain", choices=["plain", "split"])
    p.add_argument("--repeat", type=int, default=1)
    a = p.parse_args(argv)
    import numpy as np
    import torch
    from . import api, build, workloads as W
    build.build()
    if a.op == "batched_lu":
        n_list = [int(v) for v in W.batch_sizes(a.count, 16, a.nmax, seed=0)]
        mats = [W.uniform_matrix(m, a.prec, seed=W.system_seed(0, i), lda=m) for i, m in enumerate(n_list)]
        Ab = torch.from_numpy(api.pack_matrices(mats, a.prec)).cuda()
        t0 = time.perf_counter()
        for _ in range(a.repeat):
            api.ludecomp_batched(Ab, n_list, a.prec)
        torch.cuda.synchronize()
        print(f"batched_lu prec={a.prec} count={a.count} n<={a.nmax} x{a.repeat}: "
              f"{(time.perf_counter() - t0) / a.repeat * 1e3:.1f} ms per call")
        return 0
    if a.op == "batched_refine":
        import os
        n_list, kap = W.mixed_batch_spec(a.count, 64, a.nmax, 4.0, 20.0, seed=0)
        A_np, b_np = W.svd_batch(n_list, kap, seed=0, processes=len(os.sched_getaffinity(0)))
        Ab = torch.from_numpy(A_np).cuda()
        bb = torch.from_numpy(b_np).cuda()
        t0 = time.perf_counter()
        for _ in range(a.repeat):
            x, stats = api.refine_batched_blocked(Ab, 4, bb, 8, n_list, a.prec, a.update, 200)
        torch.cuda.synchronize()
        bad = int((stats[:, 3] != 0).sum())
        print(f"batched_refine inner={a.prec} update={a.update} count={a.count} n<={a.nmax} x{a.repeat}: "
              f"{(time.perf_counter() - t0) / a.repeat * 1e3:.1f} ms per call, {bad} not converged")
        return 1 if bad else 0
    if a.op == "refine":
        s = W.svd_system(a.n, 10.0, seed=0)
        A, b = s.A, s.b
    else:
        A = W.uniform_matrix(a.n, max(a.prec, 2), seed=0)
        b = W.uniform_matrix(1, 1, seed=1)[:, 0, :1]
        b = np.ones((a.prec, a.n))
    Ad = torch.from_numpy(A).cuda()
    bd = torch.from_numpy(np.ascontiguousarray(b)).cuda()
    t0 = time.perf_counter()
    for _ in range(a.repeat):
        if a.op == "lu":
            LU, piv, info = api.ludecomp(Ad, a.prec, a.update)
        elif a.op == "solve":
            LU, piv, info = api.ludecomp(Ad, a.prec)
            api.solve(LU, piv, bd, a.prec)
        elif a.op == "residual":
            x = torch.ones((8, a.n), dtype=torch.float64, device="cuda")
            api.residual(Ad, bd, x, 8)
        else:
            r = api.refine(Ad, bd, a.prec, 200, update=a.update)
            if not r.converged:
                print("refinement did not converge", file=sys.stderr)
                return 1
    torch.cuda.synchronize()
    print(f"{a.op} prec={a.prec} n={a.n} update={a.update} x{a.repeat}: "
          f"{(time.perf_counter() - t0) / a.repeat * 1e3:.1f} ms per call")
    return 0


if __name__ == "__main__":
    sys.exit(main())
