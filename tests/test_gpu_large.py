"""Past 2^31 keys (GPU): positions above the int32 range through every step
-- plan, tile sort, all merge levels and the cross-block rounds --, 2^31 + 5
int32 keys in p = 3 blocks (about 26 GB of device memory).  Checked on the
device (nondecreasing, the output's two multiset hashes equal the input's)
and at sampled ranks on the host: the key at output position k has fewer
than k+1 smaller and more than k smaller-or-equal input keys."""
import numpy as np
import pytest

from paper_1105_6040_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_more_than_2e31_keys():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_6040_gb300 import abi
    n = (1 << 31) + 5
    free, _ = torch.cuda.mem_get_info()
    if free < 40 * (1 << 30):
        pytest.skip("needs about 26 GB of free device memory")
    s = abi.Sorter(0, tile_log2=13)
    try:
        d = W.uniform_int32_torch(n, seed=77)
        rin = abi.check_keys(d)
        out = s.sort_keys(d, p=3)
        s.sync()
        rout = abi.check_keys(out)
        assert rout["first_unsorted"] == -1
        assert (rout["hash_a"], rout["hash_b"]) == (rin["hash_a"], rin["hash_b"])
        x = d.cpu().numpy()
        rng = np.random.default_rng(1)
        ks = [0, n - 1, (1 << 31) - 1, 1 << 31, (1 << 31) + 4] + [int(k) for k in rng.integers(0, n, 3)]
        vals = out[torch.tensor(ks, device="cuda")].cpu().numpy()
        del d, out
        for k, v in zip(ks, vals):
            lt = int(np.count_nonzero(x < v))
            le = int(np.count_nonzero(x <= v))
            assert lt <= k < le, (k, v, lt, le)
    finally:
        s.close()
        torch.cuda.empty_cache()
