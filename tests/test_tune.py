"""The autotuner's cache logic and knob validation (host only), and on the
GPU: tuning leaves every result bitwise unchanged."""
import numpy as np
import pytest

from paper_2107_12550_gb300 import _lib as L
from paper_2107_12550_gb300 import build as B
from paper_2107_12550_gb300 import tune as T


def test_bucket_and_key():
    assert T.bucket(1) == 16 and T.bucket(16) == 16 and T.bucket(17) == 32 and T.bucket(2048) == 2048
    assert T.key("GB300", 3, "lu", 2000) == "GB300|w3|lu|2048"


def test_cache_roundtrip_and_pick(tmp_path):
    path = str(tmp_path / "sub" / "tune.json")
    assert T.load_cache(path) == {}
    T.save_cache({"a": {"panel_width": 32}}, path)
    assert T.load_cache(path) == {"a": {"panel_width": 32}}
    best, times = T.pick_best([1, 2, 3], lambda c: {1: 0.3, 2: 0.1, 3: 0.2}[c])
    assert best == 2 and times[3] == 0.2


def test_knob_validation():
    B.build()
    lib = L.lib()
    prev = lib.mw_get_tuning(L.MW_TUNE_PANEL_WIDTH, 2)
    assert prev in (32, 64, 128)
    assert lib.mw_set_tuning(L.MW_TUNE_PANEL_WIDTH, 2, 48) == -3
    assert lib.mw_set_tuning(L.MW_TUNE_PANEL_WIDTH, 5, 64) == -2
    assert lib.mw_set_tuning(9, 2, 64) == -1
    assert lib.mw_set_tuning(L.MW_TUNE_PANEL_WIDTH, 2, 32) == prev
    assert lib.mw_get_tuning(L.MW_TUNE_PANEL_WIDTH, 2) == 32
    lib.mw_set_tuning(L.MW_TUNE_PANEL_WIDTH, 2, prev)
    assert lib.mw_set_tuning(L.MW_TUNE_BATCH_CTAS_PER_SM, 3, 0) == -3
    assert lib.mw_get_tuning(L.MW_TUNE_GEMM_TILE, 3) == 0
    assert lib.mw_set_tuning(L.MW_TUNE_GEMM_TILE, 3, 4) == -3
    assert lib.mw_set_tuning(L.MW_TUNE_GEMM_TILE, 3, -1) == -3
    assert lib.mw_set_tuning(L.MW_TUNE_GEMM_TILE, 3, 2) == 0
    assert lib.mw_set_tuning(L.MW_TUNE_GEMM_TILE, 3, 0) == 2
    assert lib.mw_get_tuning(L.MW_TUNE_BATCH_SPLIT_LEAF, 2) == 8
    assert lib.mw_set_tuning(L.MW_TUNE_BATCH_SPLIT_LEAF, 2, 12) == -3
    assert lib.mw_set_tuning(L.MW_TUNE_BATCH_SPLIT_LEAF, 2, 16) == 8
    assert lib.mw_set_tuning(L.MW_TUNE_BATCH_SPLIT_LEAF, 2, 8) == 16
    assert lib.mw_get_tuning(L.MW_TUNE_LOOKAHEAD, 3) == 1
    assert lib.mw_set_tuning(L.MW_TUNE_LOOKAHEAD, 3, 2) == -3
    assert lib.mw_set_tuning(L.MW_TUNE_LOOKAHEAD, 3, 0) == 1
    assert lib.mw_set_tuning(L.MW_TUNE_LOOKAHEAD, 3, 1) == 0
    assert lib.mw_set_tuning(L.MW_TUNE_LOOKAHEAD + 1, 3, 1) == -1
    assert lib.mw_get_tuning(L.MW_TUNE_LOOKAHEAD + 1, 3) == -1


def test_apply_from_cache(tmp_path):
    B.build()
    path = str(tmp_path / "tune.json")
    T.save_cache({T.key("FakeGPU", 4, "lu", 1000): {"panel_width": 128, "rows_per_cta": 16}}, path)
    lib = L.lib()
    old = (lib.mw_get_tuning(0, 4), lib.mw_get_tuning(1, 4))
    try:
        assert T.apply(4, 1000, path=path, gpu="FakeGPU")
        assert lib.mw_get_tuning(0, 4) == 128 and lib.mw_get_tuning(1, 4) == 16
        assert not T.apply(4, 5000, path=path, gpu="FakeGPU")
    finally:
        lib.mw_set_tuning(0, 4, old[0])
        lib.mw_set_tuning(1, 4, old[1])


def test_apply_split_knobs_and_packaged_overlay(tmp_path, monkeypatch):
    B.build()
    packaged = str(tmp_path / "packaged.json")
    user = str(tmp_path / "user.json")
    T.save_cache({T.key("FakeGPU", 2, "split_lu", 4096): {"split_leaf": 16, "rows_per_cta": 4},
                  T.key("FakeGPU", 2, "batched_split", 1024): {"batch_split_leaf": 32}}, packaged)
    T.save_cache({T.key("FakeGPU", 2, "split_lu", 4096): {"split_leaf": 32, "rows_per_cta": 8}}, user)
    monkeypatch.setattr(T, "PACKAGED", packaged)
    monkeypatch.setenv("MWLU_TUNE_CACHE", user)
    lib = L.lib()
    old = [lib.mw_get_tuning(p_, 2) for p_ in (L.MW_TUNE_SPLIT_PANEL_LEAF, L.MW_TUNE_PANEL_ROWS_PER_CTA,
                                             L.MW_TUNE_BATCH_SPLIT_LEAF)]
    try:
        # the user's entry overrides the packaged one; other entries come from the package
        assert T.apply(2, 4000, op="split_lu", gpu="FakeGPU") == {"split_leaf": 32, "rows_per_cta": 8}
        assert lib.mw_get_tuning(L.MW_TUNE_SPLIT_PANEL_LEAF, 2) == 32
        assert T.apply(2, 1000, op="batched_split", gpu="FakeGPU") == {"batch_split_leaf": 32}
        assert lib.mw_get_tuning(L.MW_TUNE_BATCH_SPLIT_LEAF, 2) == 32
        assert T.apply(2, 100, op="batched_split", gpu="FakeGPU") is None
    finally:
        for p_, v in zip((L.MW_TUNE_SPLIT_PANEL_LEAF, L.MW_TUNE_PANEL_ROWS_PER_CTA, L.MW_TUNE_BATCH_SPLIT_LEAF), old):
            lib.mw_set_tuning(p_, 2, v)


@pytest.mark.gpu
def test_tuned_lu_is_bitwise_unchanged(tmp_path):
    import torch
    import oracle
    from paper_2107_12550_gb300 import api, workloads as W
    B.build()
    lib = L.lib()
    old = (lib.mw_get_tuning(0, 3), lib.mw_get_tuning(1, 3))
    try:
        entry = T.tune_lu(3, 260, path=str(tmp_path / "t.json"), widths=(32, 64, 128), rows=(4, 32))
        assert entry["panel_width"] in (32, 64, 128)
        A = W.uniform_matrix(260, 3, seed=5)
        LUo, pivo, _ = oracle.lu(3, A)
        for nb in (32, 64, 128):
            for rpc in (1, 8, 4096):
                T.set_knob(0, 3, nb)
                T.set_knob(1, 3, rpc)
                LU, piv, info = api.ludecomp(torch.from_numpy(A).cuda(), 3)
                torch.cuda.synchronize()
                assert np.array_equal(LU.cpu().numpy()[:, :, :260], LUo[:, :, :260]), (nb, rpc)
                assert np.array_equal(piv.cpu().numpy(), pivo)
        T.set_knob(0, 3, 64)
        T.set_knob(1, 3, 8)
        for tile in (1, 2, 3, 0):
            T.set_knob(L.MW_TUNE_GEMM_TILE, 3, tile)
            LU, piv, info = api.ludecomp(torch.from_numpy(A).cuda(), 3)
            torch.cuda.synchronize()
            assert np.array_equal(LU.cpu().numpy()[:, :, :260], LUo[:, :, :260]), tile
            assert np.array_equal(piv.cpu().numpy(), pivo)
    finally:
        lib.mw_set_tuning(0, 3, old[0])
        lib.mw_set_tuning(1, 3, old[1])
        lib.mw_set_tuning(L.MW_TUNE_GEMM_TILE, 3, 0)
