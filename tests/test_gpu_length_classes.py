"""The sort phase's warp length class (GPU): blocks and segments of 1 .. 1024
keys (512 at 2048-key tiles) are sorted whole by one warp each, in a launch
before the tile sort, and get no tiles.  Every case is compared with the
oracle bit for bit, with the class on and off on the same inputs: segment
lengths at every class and tile edge, all key widths, float keys with
their total-order edge values, gathered segments, balanced blocks short
enough for the class (cross-block rounds then read the class's output),
more segments than the class's plan handles, and graph replays."""
import numpy as np
import pytest

import oracle
from paper_1105_6040_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EDGES = [0, 1, 2, 3, 31, 32, 33, 255, 511, 512, 513, 1000, 1023, 1024, 1025, 2047, 2048, 2049,
         4095, 4096, 4097, 8191, 8192, 8193, 20000]


def _bits(a):
    return a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64)


def _keys(kind, n, seed):
    if kind == "int32":
        return W.uniform_int32(n, seed=seed)
    if kind == "int32_dup":
        return (W.uniform_int32(n, seed=seed) % 5).astype(np.int32)
    if kind == "uint64":
        return W.uniform_uint64(n, seed=seed)
    if kind == "float32":
        return W.normal_float32_edges(n, seed=seed, edge_frac_pct=10)
    if kind == "float64":
        return W.uniform_float64_bits(n, seed=seed).view(np.float64)
    raise ValueError(kind)


def _dev(x):
    if x.dtype == np.uint64:
        return torch.from_numpy(x.view(np.int64)).cuda().view(torch.uint64)
    return torch.from_numpy(x).cuda()


def _host(t, like):
    if like.dtype == np.uint64:
        return t.view(torch.int64).cpu().numpy().view(np.uint64)
    return t.cpu().numpy()


def _lengths(seed):
    rng = np.random.default_rng(seed)
    lens = np.concatenate([np.repeat(EDGES, 3), W.loguniform_lengths(400, 1, 1 << 14, seed=seed)])
    return lens[rng.permutation(lens.size)].astype(np.int64)


@pytest.fixture(scope="module")
def sorters():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_6040_gb300 import abi
    from paper_1105_6040_gb300.abi import Sorter
    made = {}

    def get(tile_log2, classes):
        key = (tile_log2, classes)
        if key not in made:
            s = Sorter(0, tile_log2=tile_log2)
            abi.bs_set_option(s.h, "length_classes", classes)
            made[key] = s
        return made[key]

    yield get
    for s in made.values():
        s.close()


@pytest.mark.parametrize("tile_log2", [11, 12, 13])
@pytest.mark.parametrize("kind", ["int32", "int32_dup", "uint64", "float32", "float64"])
def test_segmented_edges_match_oracle_with_and_without_classes(sorters, tile_log2, kind):
    lens = _lengths(tile_log2 * 10 + len(kind))
    off = W.offsets_from_lengths(lens)
    x = _keys(kind, int(off[-1]), seed=tile_log2 + 7)
    want, _ = oracle.sort_segmented(x, off)
    d_off = torch.from_numpy(off).cuda()
    for classes in (1, 0):
        s = sorters(tile_log2, classes)
        s.stats(reset=True)
        got = _host(s.sort_segmented(_dev(x), d_off), x)
        counts, _ = s.stats(reset=True)
        assert np.array_equal(_bits(got), _bits(want)), (tile_log2, kind, classes)
        # the class's launch comes before the tile sort's
        assert counts["tile_sort"] == 1 + classes


def test_only_short_segments_and_empty_ones(sorters):
    """Every segment in the class (no tile at all), with empty segments
    between them; then one segment one key over the class limit."""
    rng = np.random.default_rng(3)
    lens = rng.integers(0, 1025, size=3000).astype(np.int64)
    lens[::7] = 0
    for extra in (0, 1025):
        ls = np.append(lens, extra) if extra else lens
        off = W.offsets_from_lengths(ls)
        x = _keys("int32", int(off[-1]), seed=4)
        want, _ = oracle.sort_segmented(x, off)
        got = sorters(12, 1).sort_segmented(_dev(x), torch.from_numpy(off).cuda()).cpu().numpy()
        assert np.array_equal(got, want)


def test_many_tiny_segments_beyond_the_class_plan(sorters):
    """200,000 segments (the class applies) and 300,000 (more than the
    one-kernel plan takes: every segment gets tiles again); both exact."""
    for S in (200_000, 300_000):
        lens = W.loguniform_lengths(S, 1, 64, seed=S)
        lens[::11] = 0
        off = W.offsets_from_lengths(lens)
        x = _keys("int32_dup", int(off[-1]), seed=5)
        want, _ = oracle.sort_segmented(x, off)
        got = sorters(12, 1).sort_segmented(_dev(x), torch.from_numpy(off).cuda()).cpu().numpy()
        assert np.array_equal(got, want), S


def test_gathered_short_segments(sorters):
    """Segments read from scattered places of a pool (the serving path)."""
    rng = np.random.default_rng(6)
    lens = np.concatenate([rng.integers(1, 1100, size=500), [5000, 9000, 0, 1024, 1025]]).astype(np.int64)
    pool_n = int(lens.sum()) * 2
    pool = W.normal_float32_edges(pool_n, seed=7)
    src = np.sort(rng.integers(0, pool_n - int(lens.max()), size=lens.size)).astype(np.int64)
    off = W.offsets_from_lengths(lens)
    segs = [pool[src[i]:src[i] + lens[i]] for i in range(lens.size)]
    want, _ = oracle.sort_segmented(np.concatenate(segs), off)
    for classes in (1, 0):
        s = sorters(12, classes)
        got = s.sort_gathered(torch.from_numpy(pool).cuda(), torch.from_numpy(src).cuda(),
                              torch.from_numpy(off).cuda()).cpu().numpy()
        assert np.array_equal(_bits(got), _bits(want)), classes


@pytest.mark.parametrize("n,p", [(5000, 8), (5120, 5), (5125, 5), (1 << 20, 4096), (100, 100),
                                 (7, 3), (300001, 1000)])
@pytest.mark.parametrize("persistent", [2, 0])
def test_balanced_short_blocks(sorters, n, p, persistent):
    """Balanced blocks short enough for the class (n/p up to 1024): the
    cross-block rounds merge the class's output; 5125/5 = 1025 is one key
    over, so every block takes a tile.  Three key widths, both merge forms."""
    from paper_1105_6040_gb300 import abi
    for kind in ("int32", "uint64", "float32"):
        x = _keys(kind, n, seed=n + p)
        want, _ = oracle.sort(x, p=p)
        s = sorters(12, 1)
        abi.bs_set_option(s.h, "merge_persistent", persistent)
        try:
            s.stats(reset=True)
            got = _host(s.sort_keys(_dev(x), p=p), x)
            counts, _ = s.stats(reset=True)
        finally:
            abi.bs_set_option(s.h, "merge_persistent", 1)
        assert np.array_equal(_bits(got), _bits(want)), (n, p, kind)
        # all blocks in the class: the class's launch replaces the tile sort,
        # and the plan needs no tile map
        in_class = -(-n // p) <= 1024
        assert counts["tile_sort"] == 1
        assert counts["setup"] == (1 if in_class else 2)


def test_graph_replay_with_classes(sorters):
    lens = _lengths(9)
    off = W.offsets_from_lengths(lens)
    n = int(off[-1])
    s = sorters(12, 1)
    d_in = torch.from_numpy(W.uniform_int32(n, seed=10)).cuda()
    d_off = torch.from_numpy(off).cuda()
    d_out = torch.empty_like(d_in)
    g = s.capture_segmented(d_in, d_off, d_out, max_seg_len=int(lens.max()))
    try:
        for seed in (11, 12):
            x = W.uniform_int32(n, seed=seed)
            d_in.copy_(torch.from_numpy(x))
            g.launch()
            g.sync()
            want, _ = oracle.sort_segmented(x, off)
            assert np.array_equal(d_out.cpu().numpy(), want)
    finally:
        g.close()


@pytest.mark.parametrize("direct", [1, 0])
def test_host_entry_points_with_short_blocks(sorters, direct):
    """bs_sort_keys_host with blocks in the class: with page-locked buffers
    the class's warps read and write host memory directly (the tile sort's
    role there), with pageable ones the keys are copied in and out; the
    pipelined form too."""
    from paper_1105_6040_gb300 import abi
    s = sorters(12, 1)
    abi.bs_set_option(s.h, "host_direct", direct)
    try:
        for n, p, kind in ((5000, 8, "int32"), (3000, 3, "float32"), (777, 777, "uint64"), (1 << 16, 128, "int32")):
            x = _keys(kind, n, seed=n + p + direct)
            want, _ = oracle.sort(x, p=p)
            u64 = x.dtype == np.uint64
            t = torch.from_numpy(x.view(np.int64)).view(torch.uint64) if u64 else torch.from_numpy(x)

            def host(o):
                return o.view(torch.int64).numpy().view(np.uint64) if u64 else o.numpy()

            for pinned in (True, False):
                h_in = t.pin_memory() if pinned else t.clone()
                got = host(s.sort_keys_host(h_in, p=p))
                assert np.array_equal(_bits(got), _bits(want)), (n, p, kind, pinned)
            h_in = t.pin_memory()
            h_out = torch.empty_like(h_in).pin_memory()
            s.sort_keys_host_async(h_in, h_out, p=p)
            s.sync()
            assert np.array_equal(_bits(host(h_out)), _bits(want)), (n, p, kind, "async")
    finally:
        abi.bs_set_option(s.h, "host_direct", 1)


def test_segments_bounded_by_max_len_in_the_class(sorters):
    """max_seg_len <= 1024: every segment is in the class, so the sort is the
    plan and the class's launch alone; a segment longer than the bound is
    reported as INVALID_ARG by the device check, as without the class."""
    from paper_1105_6040_gb300 import abi
    s = sorters(12, 1)
    rng = np.random.default_rng(12)
    lens = rng.integers(0, 1025, size=5000).astype(np.int64)
    off = W.offsets_from_lengths(lens)
    x = _keys("float32", int(off[-1]), seed=13)
    want, _ = oracle.sort_segmented(x, off)
    s.stats(reset=True)
    got = s.sort_segmented(_dev(x), torch.from_numpy(off).cuda(), max_seg_len=1024)
    s.sync()
    counts, _ = s.stats(reset=True)
    assert np.array_equal(_bits(got.cpu().numpy()), _bits(want))
    assert counts["tile_sort"] == 1 and counts["setup"] == 1 and counts["merge"] == 0
    bad = np.array([0, 500, 2500, 2600], dtype=np.int64)  # a 2000-key segment over the bound
    s.sort_segmented(_dev(_keys("int32", 2600, seed=14)), torch.from_numpy(bad).cuda(), max_seg_len=1024)
    with pytest.raises(abi.BsError) as e:
        s.sync()
    assert e.value.status == abi.BS_ERR_INVALID_ARG
    s.sync()  # the error was reported once and cleared
