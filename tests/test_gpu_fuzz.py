"""Seeded random combinations (GPU): each case draws an entry point (keys,
pairs, segmented keys or pairs, gathered segments), a key type and, for
pairs, a value type, a size (0 to 2^20, log-uniform, tile edges favoured),
p, the sort tile, and the library options that pick code paths (warp length
class, the merge path -- persistent forced, by size, or per pass --, merge
tile), and compares the result
with the oracle bit for bit.  The options are set on one handle and reset
between cases, so the cases also check that a handle carries no state from
one configuration to the next."""
import numpy as np
import pytest

import oracle
from paper_1105_6040_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEY_KINDS = ["int32", "uint32", "float32", "int64", "uint64", "float64"]
VAL_KINDS = ["int32", "uint32", "int64", "uint64"]


def _keys(kind, n, rng):
    seed = int(rng.integers(1 << 30))
    dup = rng.random() < 0.3  # heavy duplicates
    if kind in ("int32", "uint32"):
        x = W.uniform_int32(n, seed=seed)
        if dup:
            x = (x % 7).astype(np.int32)
        return x.view(np.uint32) if kind == "uint32" else x
    if kind == "float32":
        return W.normal_float32_edges(n, seed=seed, edge_frac_pct=5) if not dup else \
            (W.uniform_int32(n, seed=seed) % 5).astype(np.float32)
    x = W.uniform_uint64(n, seed=seed)
    if dup:
        x = x % np.uint64(9)
    if kind == "int64":
        return x.view(np.int64)
    if kind == "float64":
        return W.uniform_float64_bits(n, seed=seed).view(np.float64)
    return x


def _vals(kind, n):
    v = np.arange(n, dtype=np.int64)
    return {"int32": v.astype(np.int32), "uint32": v.astype(np.uint32), "int64": v,
            "uint64": v.astype(np.uint64)}[kind]


def _dev(x):
    if x.dtype == np.uint64:
        return torch.from_numpy(x.view(np.int64)).cuda().view(torch.uint64)
    if x.dtype == np.uint32:
        return torch.from_numpy(x.view(np.int32)).cuda().view(torch.uint32)
    return torch.from_numpy(x).cuda()


def _host(t, like):
    if like.dtype == np.uint64:
        return t.view(torch.int64).cpu().numpy().view(np.uint64)
    if like.dtype == np.uint32:
        return t.view(torch.int32).cpu().numpy().view(np.uint32)
    return t.cpu().numpy()


def _bits(a):
    return a.view({1: np.uint8, 2: np.uint16, 4: np.uint32, 8: np.uint64}[a.dtype.itemsize])


def _size(rng):
    if rng.random() < 0.3:
        T = 1 << int(rng.integers(11, 14))
        return max(0, T * int(rng.integers(1, 9)) + int(rng.integers(-2, 3)))
    return int(np.exp(rng.uniform(0, np.log(1 << 20))))


def _lengths(rng, n_target):
    lens = []
    while sum(lens) < n_target:
        r = rng.random()
        if r < 0.4:
            lens.append(int(rng.integers(0, 40)))
        elif r < 0.7:
            lens.append(int(rng.choice([1023, 1024, 1025, 4095, 4096, 4097, 8192, 8193])))
        else:
            lens.append(int(np.exp(rng.uniform(0, np.log(40000)))))
    return np.array(lens, dtype=np.int64)


@pytest.fixture(scope="module")
def handles():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_6040_gb300.abi import Sorter
    made = {}

    def get(tile_log2):
        if tile_log2 not in made:
            made[tile_log2] = Sorter(0, tile_log2=tile_log2)
        return made[tile_log2]

    yield get
    for s in made.values():
        s.close()


@pytest.mark.parametrize("case", range(160))
def test_random_case_matches_oracle(handles, case):
    from paper_1105_6040_gb300 import abi
    rng = np.random.default_rng(9000 + case)
    op = ["keys", "pairs", "segmented", "segmented_pairs", "gathered"][case % 5]
    kk = KEY_KINDS[int(rng.integers(len(KEY_KINDS)))]
    vk = VAL_KINDS[int(rng.integers(len(VAL_KINDS)))]
    tile = int(rng.integers(11, 14))
    s = handles(tile)
    opts = {"length_classes": int(rng.integers(2)), "merge_persistent": int(rng.integers(3)),
            "merge_tile_log2": int(rng.choice([0, 11, tile]))}
    for name, v in opts.items():
        abi.bs_set_option(s.h, name, v)
    try:
        what = (op, kk, vk, tile, opts)
        if op in ("keys", "pairs"):
            n = _size(rng)
            p = int(rng.choice([1, 2, 3, 7, 64, 1000, max(1, n)]))
            x = _keys(kk, n, rng)
            if op == "keys":
                want, _ = oracle.sort(x, p=min(p, max(1, n)))
                got = _host(s.sort_keys(_dev(x), p=p), x) if n else x
                assert np.array_equal(_bits(got), _bits(want)), what
            else:
                v = _vals(vk, n)
                wk, wv = oracle.sort(x, v, p=min(p, max(1, n)))
                if n:
                    ko, vo = s.sort_pairs(_dev(x), _dev(v), p=p)
                    gk, gv = _host(ko, x), _host(vo, v)
                else:
                    gk, gv = x, v
                assert np.array_equal(_bits(gk), _bits(wk)), what
                assert np.array_equal(gv, wv), what
            return
        lens = _lengths(rng, _size(rng) // 2 + 1)
        off = W.offsets_from_lengths(lens)
        n = int(off[-1])
        x = _keys(kk, n, rng)
        d_off = torch.from_numpy(off).cuda()
        if op == "segmented":
            want, _ = oracle.sort_segmented(x, off)
            got = _host(s.sort_segmented(_dev(x), d_off), x)
            assert np.array_equal(_bits(got), _bits(want)), what
        elif op == "segmented_pairs":
            v = _vals(vk, n)
            wk, wv = oracle.sort_segmented(x, off, v)
            ko, vo = s.sort_segmented(_dev(x), d_off, vals=_dev(v))
            assert np.array_equal(_bits(_host(ko, x)), _bits(wk)), what
            assert np.array_equal(_host(vo, v), wv), what
        else:  # gathered: segments read from scattered places of a pool
            pool_n = 2 * n + 16
            pool = _keys(kk, pool_n, rng)
            src = np.sort(rng.integers(0, pool_n - int(lens.max(initial=0)) + 1, size=lens.size)).astype(np.int64)
            segs = [pool[src[i]:src[i] + lens[i]] for i in range(lens.size)]
            want, _ = oracle.sort_segmented(np.concatenate(segs) if segs else pool[:0], off)
            got = _host(s.sort_gathered(_dev(pool), torch.from_numpy(src).cuda(), d_off), x)
            assert np.array_equal(_bits(got), _bits(want)), what
        s.sync()
    finally:
        for name in opts:
            abi.bs_set_option(s.h, name, {"length_classes": 1, "merge_persistent": 1, "merge_tile_log2": 0}[name])
