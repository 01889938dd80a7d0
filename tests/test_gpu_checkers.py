"""The device checkers (bs_check_keys, GPU) against the oracle's own
checkers: the two multiset hashes of every key kind equal the oracle's
hashes of the oracle's codes (two independent writings of the encodings and
of the mixes), sorted results report no offending position, and mistakes
planted on the host -- an out-of-order pair, a swapped pair of payloads --
are reported at exactly the position a host scan finds."""
import numpy as np
import pytest

import oracle
from paper_1105_6040_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_6040_gb300 import abi
    s = abi.Sorter(0)
    yield abi, s
    s.close()


def _keys(kind, n, seed):
    if kind == "int32":
        return W.uniform_int32(n, seed=seed)
    if kind == "uint32":
        return W.uniform_int32(n, seed=seed).view(np.uint32)
    if kind == "float32":
        return W.normal_float32_edges(n, seed=seed, edge_frac_pct=10)
    if kind == "int64":
        return W.uniform_uint64(n, seed=seed).view(np.int64)
    if kind == "uint64":
        return W.uniform_uint64(n, seed=seed)
    if kind == "float64":
        return W.uniform_float64_bits(n, seed=seed).view(np.float64)
    raise ValueError(kind)


def _dev(x):
    if x.dtype == np.uint64:
        return torch.from_numpy(x.view(np.int64)).cuda().view(torch.uint64)
    if x.dtype == np.uint32:
        return torch.from_numpy(x.view(np.int32)).cuda().view(torch.uint32)
    return torch.from_numpy(x).cuda()


def _first_drop(codes, off=None):
    """The host scan: smallest i with codes[i-1] > codes[i], i not a segment start."""
    i = np.nonzero(codes[1:] < codes[:-1])[0] + 1
    if off is not None:
        i = i[~np.isin(i, off)]
    return int(i[0]) if i.size else -1


KINDS = ["int32", "uint32", "float32", "int64", "uint64", "float64"]


@pytest.mark.parametrize("kind", KINDS)
def test_hashes_and_order_match_the_oracle(lib, kind):
    abi, s = lib
    n = 100_003
    x = _keys(kind, n, seed=len(kind))
    codes = oracle.encode(x)
    want = (oracle.multiset_hash(codes, 0), oracle.multiset_hash(codes, 1))
    d = _dev(x)
    r = abi.check_keys(d)
    assert (r["hash_a"], r["hash_b"]) == want
    assert r["first_unsorted"] == _first_drop(codes) and r["first_unstable"] == -1
    out = s.sort_keys(d, p=3)
    r2 = abi.check_keys(out)
    assert r2["first_unsorted"] == -1 and (r2["hash_a"], r2["hash_b"]) == want


def test_segment_starts_are_excused_and_planted_drops_found(lib):
    abi, s = lib
    lens = W.loguniform_lengths(500, 1, 5000, seed=3)
    off = W.offsets_from_lengths(lens)
    n = int(off[-1])
    x = _keys("float32", n, seed=4)
    d_off = torch.from_numpy(off).cuda()
    out = s.sort_segmented(_dev(x), d_off)
    host = out.cpu().numpy()
    codes = oracle.encode(host)
    assert abi.check_keys(out, d_off)["first_unsorted"] == -1
    # without the offsets the first segment boundary that drops is reported
    assert abi.check_keys(out)["first_unsorted"] == _first_drop(codes) != -1
    # a drop planted inside a segment: swap two unequal neighbours
    rng = np.random.default_rng(5)
    for _ in range(3):
        seg = int(rng.choice(np.nonzero(lens >= 50)[0]))
        i = int(off[seg]) + int(rng.integers(1, lens[seg] - 1))
        while codes[i - 1] == codes[i]:
            i += 1
        bad = host.copy()
        bad[i - 1], bad[i] = bad[i], bad[i - 1]
        r = abi.check_keys(torch.from_numpy(bad).cuda(), d_off)
        assert r["first_unsorted"] == _first_drop(oracle.encode(bad), off) == i
        assert (r["hash_a"], r["hash_b"]) == (oracle.multiset_hash(codes, 0), oracle.multiset_hash(codes, 1))


@pytest.mark.parametrize("idx_dtype", [np.int32, np.int64, np.uint32])
def test_stability_of_pairs_and_planted_swaps(lib, idx_dtype):
    abi, s = lib
    n = 200_000
    k = W.uniform_uint64(n, seed=6) % np.uint64(40)
    v = np.arange(n, dtype=idx_dtype)
    dk = _dev(k)
    dv = torch.from_numpy(v.view(np.int32) if idx_dtype == np.uint32 else v).cuda()
    if idx_dtype == np.uint32:
        dv = dv.view(torch.uint32)
    ko, vo = s.sort_pairs(dk, dv, p=4)
    r = abi.check_keys(ko, idx=vo)
    assert r["first_unsorted"] == -1 and r["first_unstable"] == -1
    # swap the payloads of two equal neighbouring keys
    hk = ko.view(torch.int64).cpu().numpy().view(np.uint64)
    hv = vo.view(torch.int32).cpu().numpy().view(idx_dtype) if idx_dtype == np.uint32 else vo.cpu().numpy()
    i = int(np.nonzero(hk[1:] == hk[:-1])[0][1234]) + 1
    hv2 = hv.copy()
    hv2[i - 1], hv2[i] = hv2[i], hv2[i - 1]
    dv2 = torch.from_numpy(hv2.view(np.int32) if idx_dtype == np.uint32 else hv2).cuda()
    if idx_dtype == np.uint32:
        dv2 = dv2.view(torch.uint32)
    r = abi.check_keys(ko, idx=dv2)
    assert r["first_unsorted"] == -1 and r["first_unstable"] == i


def test_full_size_sort_checked_on_the_device(lib):
    """2^26 int32 keys, p = 2: the output is sorted and has the input's hashes."""
    abi, s = lib
    d = W.uniform_int32_torch(1 << 26, seed=7)
    rin = abi.check_keys(d)
    out = s.sort_keys(d, p=2)
    rout = abi.check_keys(out)
    assert rout["first_unsorted"] == -1
    assert (rout["hash_a"], rout["hash_b"]) == (rin["hash_a"], rin["hash_b"])
    assert rin["first_unsorted"] != -1


def test_empty_and_invalid(lib):
    abi, _ = lib
    assert abi.bs_check_keys(None, 0, "int32") == {"first_unsorted": -1, "first_unstable": -1,
                                                    "hash_a": 0, "hash_b": 0}
    l = abi.load()
    assert l.bs_check_keys(None, 5, abi.DTYPES["int32"], None, 0, None, -1, None, None) == \
        abi.BS_ERR_INVALID_ARG
    d = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(abi.BsError):
        abi.bs_check_keys(d.data_ptr(), 4, "int32", d_idx=d.data_ptr(), it="float32")
