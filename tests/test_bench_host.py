"""Host-side logic of bench.py on the CPU: the batch layout it reads
systems from, the stratified sample the CPU baseline and the reference arm
time, the tensor-core work count of the split roofline, and the oracle
sample itself on small systems of the headline distribution."""
import numpy as np

import bench
from paper_2107_12550_gb300 import workloads as W


def test_stratified_sample_follows_the_order_mix():
    n_list, _ = W.mixed_batch_spec(512, 64, 1024, 4.0, 20.0, seed=0)
    ids = bench.stratified_sample(n_list, 8)
    assert len(ids) == 64 and len(set(ids)) == 64
    ns = [n_list[s] for s in ids]
    assert ns == sorted(ns)
    mean_all = np.mean(np.asarray(n_list, dtype=float) ** 3)
    mean_smp = np.mean(np.asarray(ns, dtype=float) ** 3)
    assert abs(mean_smp / mean_all - 1) < 0.05


def test_batch_system_reads_the_packed_layout():
    n_list = [3, 2]
    A = np.arange(4 * (9 + 4), dtype=float)
    b = np.arange(8 * 5, dtype=float)
    A1, b1 = bench.batch_system(A, b, n_list, 1)
    # system 1: words at 4 * 9, word c of M(i, j) at c*n*n + j*n + i
    assert A1.shape == (4, 2, 2) and A1[2, 1, 0] == 36 + 2 * 4 + 1 * 2 + 0
    assert b1.shape == (8, 2) and b1[5, 1] == 8 * 3 + 5 * 2 + 1


def test_split_trail_tile_count():
    assert bench.split_trail_mma_flops([64]) == 0
    assert bench.split_trail_mma_flops([65]) == bench.SPLIT_TILE_FLOPS
    # n = 200: m = 136 -> 2 x 9 tiles, m = 72 -> 1 x 5, m = 8 -> 1 x 1
    assert bench.split_trail_mma_flops([200]) == 24 * bench.SPLIT_TILE_FLOPS


def test_oracle_sample_on_small_systems():
    n_list, kap = [40, 64, 33], [6.0, 18.0, 12.0]
    A, b = W.svd_batch(n_list, kap, seed=3, processes=1)
    systems = [bench.batch_system(A, b, n_list, s) for s in range(3)]
    met, secs, threads = bench.oracle_batch_sample(systems)
    assert met == 3 and secs > 0 and threads >= 1
    line = bench.cpu_baseline_line(systems, "three small systems")
    assert line["kind"] == "oracle" and line["unit"] == "solves/s" and line["value"] > 0
