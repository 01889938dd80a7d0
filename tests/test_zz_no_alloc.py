"""bs_sort_keys_noalloc, through the C ABI (GPU).

The no-allocation entry point exists for callers that must not allocate GPU
memory while they sort (a latency-critical path where cudaMalloc/cudaFree can
stall the device, a plug-in inside a framework that owns all device memory);
it borrows a fixed scratch array compiled into the library instead of a
handle's cudaMalloc'ed workspace.  Each case below is sorted twice in a row
on one stream, and both outputs must equal the regular entry point's
(bs_sort_keys) and the CPU oracle's bit for bit (sorting is exact, so the
tolerance is zero).  The cases cover the capacity edges: full key capacity
with a ragged tail, p = 1024 (the largest index arrays the scratch holds),
p > n clamping, fewer keys than one tile, and in-place sorts.  Requests over
the capacity must be refused before any GPU work.  This file is named to be
collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bits(a: np.ndarray) -> np.ndarray:
    return a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64)


def test_noalloc_matches_sort_keys_and_oracle_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_1105_6040_gb300 import abi
    from paper_1105_6040_gb300 import workloads as W

    torch.cuda.set_device(0)
    s = abi.Sorter(0)
    stream = torch.cuda.current_stream().cuda_stream
    try:
        cases = [  # keys, dtype, p, in place
            (W.uniform_int32((1 << 20) - 37, seed=501), "int32", 3, False),   # full capacity, ragged
            (W.uniform_float64_bits((1 << 19) - 5, seed=502), "float64", 7, False),
            (W.uniform_int32(1 << 20, seed=503), "int32", 1024, False),      # largest index arrays
            (W.uniform_int32(1000, seed=504).view(np.uint32), "uint32", 4096, False),  # p > n
            (W.uniform_int32(100, seed=505), "int32", 1, False),            # less than one tile
            (W.uniform_int32(300001, seed=506).view(np.uint32), "uint32", 5, True),
            (W.normal_float32_edges(300000, seed=507), "float32", 2, True),
        ]
        for x, dt, p, in_place in cases:
            want_oracle, _ = oracle.sort(x, p=min(p, x.size), threads=oracle.default_threads())
            d_in = torch.from_numpy(x.copy()).cuda()
            want_lib = s.sort_keys(d_in, p=p)
            s.sync()
            outs = []
            for _ in range(2):  # two calls in a row on one stream, no sync between them
                if in_place:
                    buf = d_in.clone()
                    abi.bs_sort_keys_noalloc(buf.data_ptr(), buf.data_ptr(), x.size, dt, p, stream)
                else:
                    buf = torch.empty_like(d_in)
                    abi.bs_sort_keys_noalloc(d_in.data_ptr(), buf.data_ptr(), x.size, dt, p, stream)
                outs.append(buf)
            torch.cuda.synchronize()
            lib = _bits(want_lib.cpu().numpy())
            assert np.array_equal(lib, _bits(want_oracle)), (dt, p)
            for k, o in enumerate(outs):
                got = _bits(o.cpu().numpy())
                assert np.array_equal(got, lib), (dt, p, in_place, k)
                assert np.array_equal(got, _bits(want_oracle)), (dt, p, in_place, k)
    finally:
        s.close()


def test_noalloc_refuses_requests_over_capacity():
    from paper_1105_6040_gb300 import abi
    lib = abi.load()
    assert lib.bs_sort_keys_noalloc(1, 1, (1 << 20) + 1, abi.DTYPES["int32"], 1, None) == \
        abi.BS_ERR_TOO_LARGE
    assert lib.bs_sort_keys_noalloc(1, 1, 1 << 19, abi.DTYPES["uint64"], 1025, None) == \
        abi.BS_ERR_TOO_LARGE
    assert lib.bs_sort_keys_noalloc(None, None, 10, abi.DTYPES["int32"], 1, None) == \
        abi.BS_ERR_INVALID_ARG
