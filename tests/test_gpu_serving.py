"""Serving loop on the GPU: continuous batching of mixed int32 / float32
requests; every result equals the same request sorted alone (tolerance 0),
and a sample equals the oracle."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_serving_results_are_the_same_alone_and_in_the_mix():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_6040_gb300 import serving as S
    from paper_1105_6040_gb300.abi import Sorter

    cfg = S.ServingConfig(rate=2000, duration=0.4, lo=1 << 10, hi=1 << 18, small_max=1 << 14,
                          batch_max_keys=1 << 18, batch_max_reqs=256, streams=3,
                          pool_keys=1 << 19, keep_results=True)
    summary, reqs, ex = S.serve(cfg)
    alone = Sorter(0)
    try:
        assert summary["requests"] == len(reqs) > 400
        assert summary["batches"] < len(reqs)          # requests were batched
        assert summary["mean_batch_requests"] > 1.0
        for r in reqs:
            assert r.done >= r.launched >= r.arrival
            pool = ex.pools[r.dtype]
            want = alone.sort_keys(pool[r.src:r.src + r.n], p=1)
            alone.sync()
            assert torch.equal(r.result.view(torch.int32), want.view(torch.int32)), r.rid
        for r in reqs[::97]:
            x = ex.pools[r.dtype][r.src:r.src + r.n].cpu().numpy()
            w, _ = oracle.sort(x, p=1)
            assert np.array_equal(r.result.cpu().numpy().view(np.uint32), w.view(np.uint32))
    finally:
        alone.close()
        ex.close()


def test_gathered_segments_match_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_6040_gb300 import workloads as W
    from paper_1105_6040_gb300.abi import Sorter, bs_sync_status, BS_ERR_INVALID_ARG
    s = Sorter(0)
    try:
        pool_h = W.uniform_int32(1 << 18, seed=5)
        pool = torch.from_numpy(pool_h).cuda()
        lens = W.loguniform_lengths(200, 1, 5000, seed=6)
        src = (W.splitmix64(7, 0, 200) % np.uint64((1 << 18) - 5000)).astype(np.int64)
        off = W.offsets_from_lengths(lens)
        out = s.sort_gathered(pool, torch.from_numpy(src).cuda(), torch.from_numpy(off).cuda())
        s.sync()
        got = out.cpu().numpy()
        for i in range(200):
            seg = pool_h[src[i]:src[i] + lens[i]]
            assert np.array_equal(got[off[i]:off[i + 1]], oracle.sort(seg)[0])
        # a source range past the pool is reported, not read
        bad = src.copy()
        bad[3] = (1 << 18) - 1
        s.sort_gathered(pool, torch.from_numpy(bad).cuda(), torch.from_numpy(off).cuda())
        assert bs_sync_status(s.h) == BS_ERR_INVALID_ARG
    finally:
        s.close()


def test_tight_memory_cap_defers_and_is_respected():
    """Admission by memory: with a cap of about one largest launch's output and
    requests arriving twenty times faster, launches are deferred, the bytes in
    flight never exceed the cap, the handles' scratch reserved at start-up is
    all the library uses (it does not grow during the run), batching engages,
    and every result is still the request sorted alone."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_6040_gb300 import serving as S
    from paper_1105_6040_gb300.abi import Sorter

    # room for one largest launch (2^16 int32 keys and its batch scratch) and
    # little more: a second launch in flight beside any sizeable one waits
    cap = 4 * (1 << 16) + 4096
    cfg = S.ServingConfig(rate=40000, duration=0.1, lo=1 << 10, hi=1 << 16, small_max=1 << 12,
                          batch_max_keys=1 << 16, batch_max_reqs=64, streams=4,
                          pool_keys=1 << 18, mem_cap_bytes=cap, keep_results=True)
    summary, reqs, ex = S.serve(cfg)
    alone = Sorter(0)
    try:
        assert summary["mem_cap_bytes"] == cap
        assert summary["deferrals"] > 0
        assert 0 < summary["peak_in_flight_bytes"] <= cap
        assert summary["mean_batch_requests"] > 1.0
        assert ex.scratch_bytes() == summary["reserved_scratch_bytes"] > 0
        for r in reqs:
            assert r.done >= r.launched >= r.arrival
            want = alone.sort_keys(ex.pools[r.dtype][r.src:r.src + r.n], p=1)
            alone.sync()
            assert torch.equal(r.result.view(torch.int32), want.view(torch.int32)), r.rid
        for r in reqs[::53]:
            x = ex.pools[r.dtype][r.src:r.src + r.n].cpu().numpy()
            w, _ = oracle.sort(x, p=1)
            assert np.array_equal(r.result.cpu().numpy().view(np.uint32), w.view(np.uint32))
    finally:
        alone.close()
        ex.close()
