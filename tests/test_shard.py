"""Sharding a batch of independent systems across ranks (shard.py): the
LPT assignment, the packed subsets, and the gather of every rank's results
into the original order, with world_size 2 on the gloo backend (CPU).  On
the CPU ranks the oracle stands in for the device refinement of each
rank's subset; rank 0 checks every system's gathered x bitwise against the
oracle's refinement of that system and exactly against x* = 1 to 2^-200."""
import os
import socket
import sys
from fractions import Fraction

import numpy as np
import pytest

from paper_2107_12550_gb300 import shard
from paper_2107_12550_gb300 import workloads as W

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_lpt_assign_covers_every_system_once_and_balances():
    n_list, _ = W.mixed_batch_spec(512, 64, 1024, 4.0, 20.0, seed=0)
    for world in (1, 2, 3, 8):
        a = shard.lpt_assign(n_list, world)
        flat = sorted(s for ids in a for s in ids)
        assert flat == list(range(512))
        loads = [sum(n_list[s] ** 3 for s in ids) for ids in a]
        assert max(loads) - min(loads) <= max(n ** 3 for n in n_list)
        assert a == shard.lpt_assign(n_list, world)          # deterministic
    assert shard.lpt_assign([5, 9, 7], 2) == [[1], [2, 0]]


def test_subset_reads_the_batch_layout():
    n_list = [2, 3, 1]
    A = np.arange(4 * 14, dtype=float)
    b = np.arange(8 * 6, dtype=float)
    As, bs = shard.subset(A, b, n_list, [2, 0], 4, 8)
    assert np.array_equal(As, np.concatenate([A[4 * 13: 4 * 14], A[0: 4 * 4]]))
    assert np.array_equal(bs, np.concatenate([b[8 * 5: 8 * 6], b[0: 8 * 2]]))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


BATCH_8 = ([12, 30, 7, 25, 18, 33, 9, 21], [4.0, 12.0, 6.0, 16.0, 8.0, 20.0, 5.0, 10.0])
BATCH_2 = ([12, 30], [4.0, 12.0])


def _batch(spec):
    n_list, kap = list(spec[0]), list(spec[1])
    A, b = W.svd_batch(n_list, kap, seed=7, processes=1)
    return n_list, A, b


def _system(A, b, n_list, s):
    moff = sum(m * m for m in n_list[:s])
    voff = sum(n_list[:s])
    n = n_list[s]
    return (A[4 * moff: 4 * (moff + n * n)].reshape(4, n, n).copy(), b[8 * voff: 8 * (voff + n)].reshape(8, n).copy())


def _rank_main(rank, world, port, out, spec=BATCH_8):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2107_12550_gb300 import shard as S
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n_list, A, b = _batch(spec)
        assignment = S.lpt_assign(n_list, world)
        ids = assignment[rank]
        sub_n = [n_list[s] for s in ids]
        As, bs = S.subset(A, b, n_list, ids, 4, 8)
        xs, sts = [], []
        for k, s in enumerate(ids):                       # the oracle stands in for the device
            Ak, bk = _system(As, bs, sub_n, k)
            st, x, corr, nres, info = oracle.refine(Ak, bk, 2)
            xs.append(x.reshape(-1))
            sts.append([corr, nres, info, st])
        x_local = torch.from_numpy(np.concatenate(xs) if xs else np.zeros(0))
        st_local = torch.tensor(sts if sts else np.zeros((0, 4)), dtype=torch.int64)
        x, stats = S.gather(x_local, st_local, assignment, n_list, 8)
        if rank == 0:
            ok = True
            voff = 0
            for s, n in enumerate(n_list):
                Ak, bk = _system(A, b, n_list, s)
                st, xo, corr, nres, info = oracle.refine(Ak, bk, 2)
                xg = x[8 * voff: 8 * (voff + n)].numpy().reshape(8, n)
                ok = ok and np.array_equal(xg, xo) and list(stats[s].tolist()) == [corr, nres, info, st]
                ok = ok and all(abs(sum(Fraction(float(c)) for c in xg[:, i]) - 1) <= Fraction(1, 2 ** 200)
                                for i in range(n))
                voff += n
            out.put(("checked", ok))
        else:
            out.put(("other", x is None and stats is None))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(180)
def test_sharded_batch_gathers_every_system_over_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=150)
        assert p.exitcode == 0
    got = dict(out.get(timeout=10) for _ in range(2))
    assert got == {"checked": True, "other": True}


@pytest.mark.timeout(180)
def test_more_ranks_than_systems_leaves_a_rank_empty():
    """Three ranks, two systems: LPT gives the third rank nothing, its
    gathered parts are empty, and rank 0 still gets every system."""
    assert shard.lpt_assign(BATCH_2[0], 3) == [[1], [0], []]
    ctx = torch.multiprocessing.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 3, port, out, BATCH_2)) for r in range(3)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=150)
        assert p.exitcode == 0
    got = sorted(out.get(timeout=10) for _ in range(3))
    assert got == [("checked", True), ("other", True), ("other", True)]
