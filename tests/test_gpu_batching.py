"""Batching layer on the GPU: CUDA-graph captured sorts and the autotuner.
Results are compared with the oracle bit for bit."""
import os

import numpy as np
import pytest

import oracle
from paper_1105_6040_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sorter():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_6040_gb300.abi import Sorter
    s = Sorter(0)
    yield s
    s.close()


def test_segmented_graph_replays_with_new_offsets_and_keys(sorter):
    S, hi = 700, 1 << 14
    lens1 = W.loguniform_lengths(S, 1, hi, seed=1)
    n = int(lens1.sum())
    # a second layout with the same n and S: shuffle the lengths
    lens2 = lens1[np.random.default_rng(2).permutation(S)]
    keys1, keys2 = W.uniform_int32(n, seed=3), W.normal_float32_edges(n, seed=4).view(np.int32)
    d_in = torch.from_numpy(keys1).cuda()
    d_off = torch.from_numpy(W.offsets_from_lengths(lens1)).cuda()
    d_out = torch.empty_like(d_in)
    g = sorter.capture_segmented(d_in, d_off, d_out, max_seg_len=hi)
    try:
        for lens, keys in ((lens1, keys1), (lens2, keys2), (lens1, keys2)):
            off = W.offsets_from_lengths(lens)
            d_in.copy_(torch.from_numpy(keys))
            d_off.copy_(torch.from_numpy(off))
            g.launch()
            g.sync()
            want, _ = oracle.sort_segmented(keys, off)
            assert np.array_equal(d_out.cpu().numpy(), want)
    finally:
        g.close()


def test_segmented_graph_pairs(sorter):
    lens = W.loguniform_lengths(300, 16, 1 << 13, seed=5)
    off = W.offsets_from_lengths(lens)
    n = int(off[-1])
    k = W.uniform_uint64(n, seed=6) % np.uint64(50)
    v = W.index_payload(n)
    dk = torch.from_numpy(k.view(np.int64)).cuda().view(torch.uint64)
    dv = torch.from_numpy(v).cuda()
    ko, vo = torch.empty_like(dk), torch.empty_like(dv)
    g = sorter.capture_segmented(dk, torch.from_numpy(off).cuda(), ko, dv, vo)
    try:
        g.launch()
        g.sync()
        wk, wv = oracle.sort_segmented(k, off, v)
        assert np.array_equal(ko.view(torch.int64).cpu().numpy().view(np.uint64), wk)
        assert np.array_equal(vo.cpu().numpy(), wv)
    finally:
        g.close()


def test_keys_graph(sorter):
    x = W.uniform_int32(300001, seed=7)
    d_in = torch.from_numpy(x).cuda()
    d_out = torch.empty_like(d_in)
    g = sorter.capture_keys(d_in, d_out, p=3)
    try:
        for _ in range(2):
            g.launch()
        g.sync()
        assert np.array_equal(d_out.cpu().numpy(), oracle.sort(x, p=3)[0])
    finally:
        g.close()


def test_autotune_picks_a_config_and_caches_it(tmp_path, monkeypatch):
    from paper_1105_6040_gb300 import autotune
    from paper_1105_6040_gb300.abi import Sorter
    monkeypatch.setenv("BS_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    s = Sorter(0)
    try:
        lens = W.loguniform_lengths(200, 16, 1 << 15, seed=8)
        off = W.offsets_from_lengths(lens)
        k = W.uniform_int32(int(off[-1]), seed=9)
        dk, doff = torch.from_numpy(k).cuda(), torch.from_numpy(off).cuda()
        cfg = autotune.tune(s, "segmented", dk, offsets=doff, max_seg_len=1 << 15, repeats=1)
        assert cfg["tile_log2"] in autotune.TILE_LOG2 and cfg["merge_kernel"] in autotune.MERGE_KERNELS
        assert len(cfg["timings_ms"]) == len(autotune.CANDIDATES)
        assert os.path.exists(tmp_path / "tune.json")
        again = autotune.tune(s, "segmented", dk, offsets=doff, max_seg_len=1 << 15)
        assert again["tile_log2"] == cfg["tile_log2"]  # from the cache
        out = s.sort_segmented(dk, doff, max_seg_len=1 << 15)
        s.sync()
        assert np.array_equal(out.cpu().numpy(), oracle.sort_segmented(k, off)[0])
    finally:
        s.close()
