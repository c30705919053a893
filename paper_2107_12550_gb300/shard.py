"""A batch of independent systems sharded across the ranks of a process group.

The systems of a batch share nothing, so each rank factors and refines its
own subset with the batched calls on its own GPU, and the only collective
is the gather of the solutions and per-system statistics at the end.

* ``lpt_assign(n_list, world)``: longest-processing-time-first on the work
  estimate n^3 (the LU's 2/3 n^3 multiword operations dominate the step):
  systems in decreasing order of n (ties by index), each to the rank with
  the least work so far (ties to the lowest rank).  Every rank computes the
  same assignment from the orders alone.
* ``subset(A, b, n_list, ids, a_words, b_words)``: the packed batch arrays
  (the layout of include/mwlu.h) of the systems ``ids``, in that order.
* ``gather(x_local, stats_local, assignment, n_list, x_words, dst)``: on
  rank ``dst`` the full packed x and the (count, 4) statistics in the
  original order; None elsewhere.  The flattened local results are padded
  to a common length and exchanged with one all_gather per array, which
  every backend supports (gloo on CPU tensors, NCCL on CUDA tensors).
* ``refine_batched_sharded(...)``: one rank's part of the batched mixed
  precision refinement: its subset to its GPU, the blocked batched
  refinement, then the gather.
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np


def lpt_assign(n_list: Sequence[int], world: int) -> List[List[int]]:
    """Per rank, the indices of its systems (in decreasing order of n)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(n_list)), key=lambda s: (-int(n_list[s]), s))
    load = [0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for s in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(s)
        load[r] += int(n_list[s]) ** 3
    return out


def _offsets(n_list):
    n = np.asarray(n_list, dtype=np.int64)
    return np.concatenate([[0], np.cumsum(n * n)]), np.concatenate([[0], np.cumsum(n)])


def subset(A, b, n_list: Sequence[int], ids: Sequence[int], a_words: int, b_words: int):
    """Packed (A, b) of the systems ``ids`` (numpy arrays or torch tensors,
    flat, in the batch layout)."""
    moff, voff = _offsets(n_list)
    As = [A[a_words * int(moff[s]): a_words * int(moff[s + 1])] for s in ids]
    bs = [b[b_words * int(voff[s]): b_words * int(voff[s + 1])] for s in ids]
    if isinstance(A, np.ndarray):
        return np.concatenate(As) if As else A[:0], np.concatenate(bs) if bs else b[:0]
    import torch
    return (torch.cat(As) if As else A[:0]), (torch.cat(bs) if bs else b[:0])


def _all_gather_padded(t, dist, group=None):
    import torch
    world = dist.get_world_size(group)
    n = torch.tensor([t.numel()], dtype=torch.int64, device=t.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    m = int(max(int(v.item()) for v in sizes))
    pad = torch.zeros(m, dtype=t.dtype, device=t.device)
    pad[: t.numel()] = t.reshape(-1)
    parts = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return [p[: int(sz.item())] for p, sz in zip(parts, sizes)]


def gather(x_local, stats_local, assignment: Sequence[Sequence[int]], n_list: Sequence[int], x_words: int,
           dst: int = 0, group=None):
    """(x, stats) of the whole batch on rank dst, in the original order, as
    tensors on the local results' device; (None, None) on other ranks."""
    import torch
    import torch.distributed as dist
    xs = _all_gather_padded(x_local.reshape(-1), dist, group)
    ss = _all_gather_padded(stats_local.reshape(-1), dist, group)
    if dist.get_rank(group) != dst:
        return None, None
    _, voff = _offsets(n_list)
    x = torch.zeros(x_words * int(voff[-1]), dtype=x_local.dtype, device=x_local.device)
    stats = torch.zeros((len(n_list), 4), dtype=stats_local.dtype, device=stats_local.device)
    for r, ids in enumerate(assignment):
        off = 0
        st = ss[r].reshape(-1, 4)
        for k, s in enumerate(ids):
            m = x_words * int(n_list[s])
            x[x_words * int(voff[s]): x_words * int(voff[s]) + m] = xs[r][off: off + m]
            off += m
            stats[s] = st[k]
    return x, stats


def refine_batched_sharded(A_host, a_words: int, b_host, b_words: int, n_list, inner_prec="dd", update="split",
                           target_bits: int = 200, *, x_words: int = 8, dst: int = 0, group=None):
    """This rank's share of the batched refinement of the whole batch
    (host arrays A_host, b_host in the batch layout, the same on every
    rank), followed by the gather: (x, stats) on rank dst, (None, None)
    elsewhere.  Each rank uses its current CUDA device."""
    import torch
    import torch.distributed as dist
    from . import api
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    assignment = lpt_assign(n_list, world)
    ids = assignment[rank]
    sub_n = [int(n_list[s]) for s in ids]
    A_s, b_s = subset(A_host, b_host, n_list, ids, a_words, b_words)
    if sub_n:
        A_d = torch.as_tensor(A_s).cuda()
        b_d = torch.as_tensor(b_s).cuda()
        x_d, st_d = api.refine_batched_blocked(A_d, a_words, b_d, b_words, sub_n, inner_prec, update, target_bits,
                                               x_words=x_words)
    else:
        x_d = torch.zeros(0, dtype=torch.float64, device="cuda")
        st_d = torch.zeros((0, 4), dtype=torch.int64, device="cuda")
    return gather(x_d, st_d, assignment, n_list, x_words, dst=dst, group=group)
