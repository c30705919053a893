"""The multi-GPU path of bench.py is replicas: each rank solves its own
system and only (time, systems solved) cross ranks, as the max time and the
summed count.  Checked here with world_size 2 on the gloo backend (CPU)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, solved = bench.combine_ranks(10.0 * (rank + 1), 3 + rank, "cpu")
        out.put((rank, ms, solved))
        world_, rank_, local_ = bench.dist_setup(None)
        out.put(("env", rank, world_, rank_))
    finally:
        dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_replicas_combine_over_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    env_backup = {k: os.environ.get(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    for r, p in enumerate(procs):
        os.environ.update({"WORLD_SIZE": "2", "RANK": str(r), "LOCAL_RANK": str(r)})
        p.start()
    for k, v in env_backup.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v
    for p in procs:
        p.join(timeout=90)
        assert p.exitcode == 0
    got = [out.get(timeout=10) for _ in range(4)]
    combined = sorted(g for g in got if g[0] != "env")
    assert combined == [(0, 20.0, 7), (1, 20.0, 7)]
    envs = sorted(g[1:] for g in got if g[0] == "env")
    assert envs == [(0, 2, 0), (1, 2, 1)]


def test_single_process_combine_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(12.5, 4, "cpu") == (12.5, 4)
