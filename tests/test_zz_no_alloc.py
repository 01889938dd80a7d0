"""bs_sort_keys_noalloc, through the C ABI, against bs_sort_keys (GPU).

The no-allocation entry point exists for callers that must not allocate GPU
memory while they sort; it borrows a fixed scratch array compiled into the
library instead of a handle's cudaMalloc'ed workspace.  Two calls in a row
must each give exactly the regular entry point's output (sorting is exact, so
the tolerance is zero), and requests over the array's capacity must be
refused before any GPU work.  This file is named to be collected last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_matches_sort_keys_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_6040_gb300 import abi
    from paper_1105_6040_gb300 import workloads as W

    torch.cuda.set_device(0)
    s = abi.Sorter(0)
    stream = torch.cuda.current_stream().cuda_stream
    try:
        cases = [
            (W.uniform_int32((1 << 20) - 37, seed=501), "int32", 3),     # full capacity, ragged
            (W.uniform_float64_bits((1 << 19) - 5, seed=502), "float64", 7),
        ]
        for x, dt, p in cases:
            d_in = torch.from_numpy(x).cuda()
            want = s.sort_keys(d_in, p=p)
            got = torch.empty_like(d_in)
            abi.bs_sort_keys_noalloc(d_in.data_ptr(), got.data_ptr(), x.size, dt, p, stream)
            torch.cuda.synchronize()
            s.sync()
            bits = np.uint32 if x.dtype.itemsize == 4 else np.uint64
            assert np.array_equal(got.cpu().numpy().view(bits), want.cpu().numpy().view(bits)), dt
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
