"""The sharded batched refinement (shard.refine_batched_sharded) on the GPU
in a one-rank process group: its gathered x and statistics equal the
unsharded blocked batched refinement's, bitwise."""
import os
import socket

import pytest

from paper_2107_12550_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_one_rank_shard_equals_the_batched_call():
    import torch.distributed as dist
    from paper_2107_12550_gb300 import api, shard
    from paper_2107_12550_gb300 import build as B
    B.build()
    n_list, kap = W.mixed_batch_spec(16, 64, 300, 4.0, 20.0, seed=3)
    A, b = W.svd_batch(n_list, kap, seed=3, processes=2)
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("nccl", rank=0, world_size=1, device_id=torch.device("cuda", 0))
    try:
        x, st = shard.refine_batched_sharded(A, 4, b, 8, n_list)
        torch.cuda.synchronize()
    finally:
        dist.destroy_process_group()
    xr, str_ = api.refine_batched_blocked(torch.from_numpy(A).cuda(), 4, torch.from_numpy(b).cuda(), 8, n_list,
                                          "dd", "split", 200)
    torch.cuda.synchronize()
    assert torch.equal(x, xr) and torch.equal(st, str_)
    assert (st[:, 3] == 0).all()
