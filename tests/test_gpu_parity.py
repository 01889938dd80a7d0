"""CUDA path against the CPU oracle, bit for bit, through the C ABI (GPU only).

Sorting has one correct output (keys-only) and one correct stable output
(pairs), so every comparison here is exact: tolerance 0.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1105_6040_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

T = 4096  # default tile


@pytest.fixture(scope="module")
def sorter():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_6040_gb300.abi import Sorter
    s = Sorter(0)
    yield s
    s.close()


def _bits(a: np.ndarray) -> np.ndarray:
    return a.view(np.uint32 if a.dtype.itemsize == 4 else np.uint64)


def _to_dev(a: np.ndarray):
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32)).cuda().view(torch.uint32)
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64)).cuda().view(torch.uint64)
    return torch.from_numpy(a).cuda()


def _to_host(t) -> np.ndarray:
    if t.dtype == torch.uint32:
        return t.view(torch.int32).cpu().numpy().view(np.uint32)
    if t.dtype == torch.uint64:
        return t.view(torch.int64).cpu().numpy().view(np.uint64)
    return t.cpu().numpy()


def gpu_keys(sorter, x, p):
    out = sorter.sort_keys(_to_dev(x), p=p)
    sorter.sync()
    return _to_host(out)


def check_keys(sorter, x, p):
    got = gpu_keys(sorter, x, p)
    want, _ = oracle.sort(x, p=p, threads=os.cpu_count() or 1)
    assert np.array_equal(_bits(got), _bits(want)), (x.dtype, x.size, p)


# ------------------------------------------------------------------ int32 keys, sizes x p

SIZES = [1, 2, 3, 100, T - 1, T, T + 1, 3 * T + 17, 2 * T * 8 + 5, 65536 + 123]


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("p", [1, 2, 3, 7, 64])
def test_int32_uniform_sizes(sorter, n, p):
    check_keys(sorter, W.uniform_int32(n, seed=n * 131 + p), p)


@pytest.mark.parametrize("dist", ["uniform", "sorted", "reverse", "dup16"])
@pytest.mark.parametrize("p", [1, 2, 5, 64, 4096])
def test_int32_distributions_2e18(sorter, dist, p):
    check_keys(sorter, W.int32_keys(dist, 1 << 18, seed=7), p)


def test_pr1_config_2e20_p2(sorter):
    """2^20 uniform int32 keys, p = 2 (the paper's dual-core decomposition)."""
    check_keys(sorter, W.uniform_int32(1 << 20, seed=W.DEFAULT_SEED), 2)


@pytest.mark.parametrize("n,p", [(1, 5), (7, 7), (10, 3), (5000, 5000), (5000, 6000), (9000, 4500)])
def test_degenerate_blocks(sorter, n, p):
    """p close to or above n: blocks of one or two keys (p > n clamps to n)."""
    check_keys(sorter, W.uniform_int32(n, seed=3) % 97, p)


def test_empty_is_noop(sorter):
    x = torch.empty(0, dtype=torch.int32, device="cuda")
    out = sorter.sort_keys(x, p=3)
    sorter.sync()
    assert out.numel() == 0


# ------------------------------------------------------------------ other key dtypes

@pytest.mark.parametrize("maker", [
    lambda n: W.uniform_int32(n, 11).view(np.uint32),
    lambda n: W.normal_float32_edges(n, 12),
    lambda n: W.uniform_float32_bits(n, 13),          # NaNs, infinities, subnormals
    lambda n: W.uniform_uint64(n, 14).view(np.int64),
    lambda n: W.uniform_uint64(n, 15),
    lambda n: W.uniform_float64_bits(n, 16),
    lambda n: W.zipf_uint64(n, 17),
], ids=["uint32", "float32_normal_edges", "float32_bits", "int64", "uint64", "float64_bits",
        "uint64_zipf"])
@pytest.mark.parametrize("n,p", [(T + 3, 1), (50001, 3), (1 << 17, 16)])
def test_key_dtypes(sorter, maker, n, p):
    check_keys(sorter, maker(n), p)


def test_float_total_order_specials(sorter):
    words = [int(l.split()[0], 16) for l in open(os.path.join(os.path.dirname(__file__), "golden",
                                                               "float32_total_order.txt"))
             if l.strip() and not l.startswith("#")]
    w = np.array(words, dtype=np.uint32)
    rng = np.random.default_rng(5)
    x = np.tile(w, 300)[rng.permutation(300 * w.size)].view(np.float32)
    got = gpu_keys(sorter, x, 4)
    assert np.array_equal(_bits(got), np.repeat(w, 300))


_LARGEST = {"int32": (W.uniform_int32, np.int32, 0x7FFFFFFF),
            "uint32": (lambda n, sd: W.uniform_int32(n, sd).view(np.uint32), np.uint32, 0xFFFFFFFF),
            "uint64": (W.uniform_uint64, np.uint64, 0xFFFFFFFFFFFFFFFF),
            "float32_nan": (lambda n, sd: W.uniform_int32(n, sd).view(np.uint32), np.uint32, 0x7FFFFFFF)}


@pytest.mark.parametrize("kind", list(_LARGEST))
@pytest.mark.parametrize("frac", [0.5, 0.97, 1.0])
@pytest.mark.parametrize("n,p", [(T - 1, 1), (3 * T + 17, 2), (1 << 17, 8)])
def test_largest_code_keys(sorter, kind, frac, n, p):
    # keys whose code is the largest one -- the value padding slots and
    # exhausted list heads read as in the tile sort and the merge passes
    make, dt, top = _LARGEST[kind]
    x = make(n, 23).astype(dt)
    rng = np.random.default_rng(24)
    x[rng.random(n) < frac] = dt(top)
    if kind == "float32_nan":
        x = x.view(np.float32)  # +NaN with every payload bit set is the largest float32 code
    check_keys(sorter, x, p)


# ------------------------------------------------------------------ stable pairs

@pytest.mark.parametrize("keys", ["uniform", "zipf", "dup"])
@pytest.mark.parametrize("n,p", [(T - 1, 1), (3 * T + 5, 2), (1 << 18, 8), (100003, 7)])
def test_pairs_uint64_index_payload_stable(sorter, keys, n, p):
    k = {"uniform": lambda: W.uniform_uint64(n, 21), "zipf": lambda: W.zipf_uint64(n, 22),
         "dup": lambda: W.uniform_uint64(n, 23) % np.uint64(5)}[keys]()
    v = W.index_payload(n)
    ko, vo = sorter.sort_pairs(_to_dev(k), _to_dev(v), p=p)
    sorter.sync()
    wk, wv = oracle.sort(k, v, p=p, threads=os.cpu_count() or 1)
    assert np.array_equal(_to_host(ko), wk)
    assert np.array_equal(_to_host(vo), wv)


@pytest.mark.parametrize("kmaker,vdtype", [
    (lambda n: W.uniform_int32(n, 31) % 1000, np.float32),
    (lambda n: W.normal_float32_edges(n, 32), np.int64),
    (lambda n: (W.uniform_uint64(n, 33) % np.uint64(77)).view(np.int64), np.int32),
    (lambda n: W.uniform_float64_bits(n, 34), np.float64),
], ids=["i32_f32", "f32_i64", "i64_i32", "f64_f64"])
def test_pairs_mixed_dtypes(sorter, kmaker, vdtype):
    n = 40000
    k = kmaker(n)
    v = W.uniform_uint64(n, 35).astype(np.uint64).view(np.int64)[:n].astype(vdtype) \
        if vdtype != np.float64 else W.uniform_float64_bits(n, 36)
    ko, vo = sorter.sort_pairs(_to_dev(k), _to_dev(v), p=3)
    sorter.sync()
    wk, wv = oracle.sort(k, v, p=3)
    assert np.array_equal(_bits(_to_host(ko)), _bits(wk))
    assert np.array_equal(_bits(_to_host(vo)), _bits(wv))


# ------------------------------------------------------------------ segmented

@pytest.mark.parametrize("with_vals", [False, True])
@pytest.mark.parametrize("case", ["mixed", "tiny", "one", "with_empty", "loguniform"])
def test_segmented(sorter, case, with_vals):
    lens = {
        "mixed": np.array([5, 0, T, T + 1, 1, 3 * T - 7, 17, 0, 9 * T + 3, 2]),
        "tiny": np.full(3000, 3),
        "one": np.array([100000]),
        "with_empty": np.array([0, 0, 7, 0, 0, 0, T * 2, 0]),
        "loguniform": W.loguniform_lengths(300, 16, 1 << 16, seed=41),
    }[case].astype(np.int64)
    off = W.offsets_from_lengths(lens)
    n = int(off[-1])
    k = W.uniform_int32(n, seed=42) % 5000
    v = W.index_payload(n) if with_vals else None
    res = sorter.sort_segmented(_to_dev(k), torch.from_numpy(off).cuda(),
                                None if v is None else _to_dev(v))
    sorter.sync()
    wk, wv = oracle.sort_segmented(k, off, v)
    if with_vals:
        ko, vo = res
        assert np.array_equal(_to_host(ko), wk) and np.array_equal(_to_host(vo), wv)
    else:
        assert np.array_equal(_to_host(res), wk)


def test_segmented_max_len_hint(sorter):
    lens = W.loguniform_lengths(500, 16, 1 << 14, seed=43)
    off = W.offsets_from_lengths(lens)
    k = W.uniform_int32(int(off[-1]), seed=44)
    res = sorter.sort_segmented(_to_dev(k), torch.from_numpy(off).cuda(), max_seg_len=int(lens.max()))
    sorter.sync()
    assert np.array_equal(_to_host(res), oracle.sort_segmented(k, off)[0])


def test_segmented_bad_offsets_reported_not_faulted(sorter):
    from paper_1105_6040_gb300 import abi
    k = _to_dev(W.uniform_int32(1000, 1))
    for bad in ([0, 600, 400, 1000], [0, 500, 999], [5, 500, 1000], [0, 500, 2000]):
        sorter.sort_segmented(k, torch.tensor(bad, dtype=torch.int64, device="cuda"))
        assert abi.bs_sync_status(sorter.h) == abi.BS_ERR_INVALID_ARG
    # a segment longer than the promised bound
    sorter.sort_segmented(k, torch.tensor([0, 1000], dtype=torch.int64, device="cuda"), max_seg_len=10)
    assert abi.bs_sync_status(sorter.h) == abi.BS_ERR_INVALID_ARG
    sorter.sync()  # the handle is usable again


# ------------------------------------------------------------------ in place, tiles, streams

def test_in_place(sorter):
    x = W.uniform_int32(3 * T + 11, 51)
    t = _to_dev(x)
    sorter.sort_keys(t, out=t, p=3)
    sorter.sync()
    assert np.array_equal(_to_host(t), np.sort(x))
    k, v = W.uniform_uint64(20000, 52) % np.uint64(9), W.index_payload(20000)
    tk, tv = _to_dev(k), _to_dev(v)
    sorter.sort_pairs(tk, tv, kout=tk, vout=tv, p=2)
    sorter.sync()
    wk, wv = oracle.sort(k, v, p=2)
    assert np.array_equal(_to_host(tk), wk) and np.array_equal(_to_host(tv), wv)


@pytest.mark.parametrize("tile_log2", [11, 12, 13])
def test_tile_shapes(tile_log2):
    from paper_1105_6040_gb300.abi import Sorter
    s = Sorter(0, tile_log2=tile_log2)
    try:
        for n, p in ((70001, 3), (1 << 17, 1)):
            check_keys(s, W.uniform_int32(n, n + tile_log2), p)
        k, v = W.zipf_uint64(30001, 61), W.index_payload(30001)
        ko, vo = s.sort_pairs(_to_dev(k), _to_dev(v), p=5)
        s.sync()
        wk, wv = oracle.sort(k, v, p=5)
        assert np.array_equal(_to_host(ko), wk) and np.array_equal(_to_host(vo), wv)
    finally:
        s.close()


def test_side_stream(sorter):
    x = W.uniform_int32(100000, 71)
    t = _to_dev(x)
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        out = sorter.sort_keys(t, p=4, stream=st)
    st.synchronize()
    assert np.array_equal(_to_host(out), np.sort(x))


def test_host_buffer_entry_point(sorter):
    x = W.uniform_int32(300001, 81)
    h = torch.from_numpy(x).pin_memory()
    out = sorter.sort_keys_host(h, p=2)
    assert np.array_equal(out.numpy(), oracle.sort(x, p=2)[0])


@pytest.mark.parametrize("direct", [1, 0])
@pytest.mark.parametrize("case", ["one_tile", "p2", "p8_float", "uint64_p3", "oddeven_p5", "in_place",
                                  "pageable", "large_2e25", "large_float_in_place"])
def test_host_entry_direct_and_copy(direct, case):
    """bs_sort_keys_host gives the oracle's output whether the kernels address
    the page-locked host buffers directly or copy through device memory."""
    from paper_1105_6040_gb300 import abi
    from paper_1105_6040_gb300.abi import Sorter
    s = Sorter(0)
    try:
        abi.bs_set_option(s.h, "host_direct", direct)
        p, dt = 2, "int32"
        if case == "one_tile":
            x, p = W.uniform_int32(3000, 90), 1
        elif case == "p2":
            x = W.uniform_int32(300001, 91)
        elif case == "p8_float":
            x, p = W.normal_float32_edges(1 << 20, 92), 8
        elif case == "uint64_p3":
            x, p = W.uniform_uint64(200003, 93), 3
        elif case == "oddeven_p5":
            abi.bs_set_option(s.h, "merge_schedule", 1)
            x, p = W.uniform_int32(100003, 94), 5
        elif case == "large_2e25":  # many tiles, ragged blocks
            x, p = W.uniform_int32((1 << 25) + 12345, 96), 3
        elif case == "large_float_in_place":
            x, p = W.normal_float32_edges((1 << 26) + 7, 97), 2
        else:
            x = W.dup16_int32(250000, 95)
        want = oracle.sort(x, p=p)[0]
        if case == "pageable":
            h_in, h_out = torch.from_numpy(x.copy()), torch.empty(x.size, dtype=torch.from_numpy(x).dtype)
        else:
            h_in = torch.from_numpy(x.copy()).pin_memory()
            h_out = h_in if case.endswith("in_place") else torch.empty_like(h_in).pin_memory()
        s.sort_keys_host(h_in, h_out, p=p)
        assert np.array_equal(_bits(h_out.numpy()), _bits(want))
    finally:
        s.close()


@pytest.mark.parametrize("slots", [3, 2])
def test_host_async_pipeline(slots):
    """bs_sort_keys_host_async: six calls in flight on one handle (its two
    or three slots of input and output buffers used in turn, copies
    overlapping sorts), interleaved with
    calls on a second handle and stream; int32, float32 and uint64 keys,
    growing sizes (a buffer regrown between calls), one call in place and
    one from pageable memory.  Every result is the oracle's."""
    from paper_1105_6040_gb300 import abi
    from paper_1105_6040_gb300.abi import Sorter
    sorters = [Sorter(0), Sorter(0)]
    for sr in sorters:
        abi.bs_set_option(sr.h, "host_slots", slots)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    try:
        xs = [W.uniform_int32((1 << 21) + 13, 111), W.normal_float32_edges(1 << 22, 112),
              W.uniform_uint64(300007, 113), W.uniform_int32((1 << 23) + 5, 114),
              W.dup16_int32(1 << 20, 115), W.uniform_float32_bits((1 << 22) + 99, 116),
              W.uniform_int32(5000, 117), W.uniform_uint64((1 << 21) + 1, 118)]
        ps = [2, 3, 1, 8, 4, 2, 1, 5]
        ins = [torch.from_numpy(x.copy()) if k == 4 else torch.from_numpy(x.copy()).pin_memory()
               for k, x in enumerate(xs)]
        outs = [ins[k] if k == 3 else torch.empty_like(ins[k]).pin_memory() for k in range(len(xs))]
        for k in range(len(xs)):
            j = 1 if k in (2, 5) else 0  # most calls on the first handle, back to back
            sorters[j].sort_keys_host_async(ins[k], outs[k], p=ps[k], stream=streams[j])
        for sr in sorters:
            sr.sync()
        for k in range(len(xs)):
            want = oracle.sort(xs[k], p=ps[k])[0]
            assert np.array_equal(_bits(outs[k].numpy()), _bits(want)), k
    finally:
        for sr in sorters:
            sr.close()


def test_invalid_args(sorter):
    from paper_1105_6040_gb300 import abi
    t = torch.zeros(10, dtype=torch.int32, device="cuda")
    with pytest.raises(abi.BsError) as e:
        abi.bs_sort_keys(sorter.h, t.data_ptr(), t.data_ptr(), 10, "int32", -1)
    assert e.value.status == abi.BS_ERR_INVALID_ARG
    with pytest.raises(abi.BsError) as e:
        abi.bs_sort_keys(sorter.h, t.data_ptr(), t.data_ptr(), 10, "none", 1)
    assert e.value.status == abi.BS_ERR_UNSUPPORTED_DTYPE
    with pytest.raises(abi.BsError) as e:
        abi.bs_sort_pairs(sorter.h, t.data_ptr(), t.data_ptr(), t.data_ptr(), t.data_ptr(), 10,
                          "int32", "none", 1)
    assert e.value.status == abi.BS_ERR_UNSUPPORTED_DTYPE


def test_launch_stats_count_passes(sorter):
    """1 tile-sort pass + 7 in-block levels (2^19 / 4096 = 2^7 tiles) + 1 cross
    round: one persistent merge launch when forced, 8 partition + 8 merge
    launches per pass otherwise -- and by default at this size, too small
    for every resident CTA to get a batch of a level; the algorithmic bytes
    are the same."""
    from paper_1105_6040_gb300 import abi
    n = 1 << 20
    for persistent, merges, parts in ((2, 1, 0), (0, 8, 8), (1, 8, 8)):
        abi.bs_set_option(sorter.h, "merge_persistent", persistent)
        sorter.stats(reset=True)
        abi.bs_set_option(sorter.h, "count_bytes", 1)
        try:
            sorter.sort_keys(_to_dev(W.uniform_int32(n, 91)), p=2)
            counts, byts = sorter.stats(reset=True)
        finally:
            abi.bs_set_option(sorter.h, "count_bytes", 0)
            abi.bs_set_option(sorter.h, "merge_persistent", 1)
        assert counts["tile_sort"] == 1 and counts["merge"] == merges and counts["partition"] == parts
        assert byts["tile_sort"] == 2 * 4 * n and byts["merge"] == 8 * 2 * 4 * n
    # counting off (the default): the same sort adds no bytes
    sorter.sort_keys(_to_dev(W.uniform_int32(n, 92)), p=2)
    counts, byts = sorter.stats(reset=True)
    assert counts["merge"] == 8 and byts["tile_sort"] == 0 and byts["merge"] == 0


@pytest.mark.parametrize("tile_log2,merge_tile_log2", [(12, 0), (13, 11), (11, 11), (13, 13)])
def test_persistent_merge_matches_per_pass_and_oracle(tile_log2, merge_tile_log2):
    """The persistent merge (every level in one launch, tiles waiting on the
    pairs they read) against the per-pass kernels and the oracle: balanced
    blocks at p up to 4096 and not powers of two, keys of every width, stable
    pairs, segmented batches whose short segments leave most upper-level tiles
    inactive, merge-only runs; each case run three times on one handle."""
    from paper_1105_6040_gb300 import abi
    from paper_1105_6040_gb300.abi import Sorter
    per = Sorter(0, tile_log2=tile_log2, merge_tile_log2=merge_tile_log2)
    abi.bs_set_option(per.h, "merge_persistent", 0)
    pst = Sorter(0, tile_log2=tile_log2, merge_tile_log2=merge_tile_log2)
    abi.bs_set_option(pst.h, "merge_persistent", 2)  # these sizes would run per pass by default
    try:
        for n, p in ((1, 1), (T - 1, 1), (3 * T + 7, 2), (100003, 3), (1 << 18, 6), (262139, 4096),
                     ((1 << 20) + 5, 7), (1 << 21, 1)):
            for x in (W.uniform_int32(n, n + p), W.uniform_uint64(n, n + p + 1)):
                want, _ = oracle.sort(x, p=min(p, n), threads=8)
                a = gpu_keys(per, x, p)
                assert np.array_equal(_bits(a), _bits(want)), (n, p, "per-pass")
                for _ in range(3):
                    b = gpu_keys(pst, x, p)
                    assert np.array_equal(_bits(b), _bits(want)), (n, p, "persistent")
        for kmaker, vmaker in ((lambda n: W.uniform_int32(n, 8) % 300, W.index_payload),
                               (lambda n: W.zipf_uint64(n, 7), lambda n: W.uniform_uint64(n, 9))):
            n, p = 300007, 5
            k, v = kmaker(n), vmaker(n)
            wk, wv = oracle.sort(k, v, p=p)
            for _ in range(3):
                ko, vo = pst.sort_pairs(_to_dev(k), _to_dev(v), p=p)
                pst.sync()
                assert np.array_equal(_bits(_to_host(ko)), _bits(wk))
                assert np.array_equal(_bits(_to_host(vo)), _bits(wv))
        lens = W.loguniform_lengths(3000, 1, 1 << 17, seed=79)
        off = W.offsets_from_lengths(lens)
        k = W.uniform_int32(int(off[-1]), seed=80)
        want = oracle.sort_segmented(k, off)[0]
        for _ in range(3):
            res = pst.sort_segmented(_to_dev(k), torch.from_numpy(off).cuda())
            pst.sync()
            assert np.array_equal(_to_host(res), want)
        # merge phase only: 37 caller-sorted runs of uneven length, some empty
        rl = W.loguniform_lengths(37, 1, 1 << 15, seed=81)
        rl[[3, 17]] = 0
        roff = W.offsets_from_lengths(rl)
        x = W.uniform_int32(int(roff[-1]), seed=82)
        runs = np.concatenate([np.sort(x[roff[i]:roff[i + 1]]) for i in range(len(rl))])
        for _ in range(3):
            out = pst.merge_runs(_to_dev(runs), [int(v) for v in roff])
            pst.sync()
            assert np.array_equal(_to_host(out), np.sort(x))
    finally:
        per.close()
        pst.close()


# ------------------------------------------------------------------ full sizes

def test_2e26_int32_dup16_p4096_full_compare(sorter):
    x = W.dup16_int32(1 << 26, seed=101)
    check_keys(sorter, x, 4096)


@pytest.mark.parametrize("dist,log2n", [("uniform", 27), ("zipf", 26)])
def test_pairs_uint64_int32_full_size(sorter, dist, log2n):
    """The stable-pairs workload at full size (Zipf at 2^26 to bound the host
    generator's time): the output is the stable sort iff the payload is a
    permutation, every key travelled with its payload, the keys are
    nondecreasing and equal keys keep their payload order (fast checks on the
    GPU); then keys and values are compared element by element with the
    oracle's stable sort."""
    n = 1 << log2n
    k = W.uniform_uint64(n, seed=W.DEFAULT_SEED) if dist == "uniform" else W.zipf_uint64(n, seed=W.DEFAULT_SEED)
    v = W.index_payload(n)
    dk, dv = _to_dev(k), _to_dev(v)
    ko, vo = sorter.sort_pairs(dk, dv, p=2)
    sorter.sync()
    idx = vo.long()
    assert bool((torch.bincount(idx, minlength=n) == 1).all())
    assert torch.equal(ko.view(torch.int64), dk.view(torch.int64)[idx])
    code = ko.view(torch.int64) ^ torch.tensor(-(1 << 63), dtype=torch.int64, device="cuda")
    assert bool((code[1:] >= code[:-1]).all())
    eq = code[1:] == code[:-1]
    assert bool((vo[1:][eq] > vo[:-1][eq]).all())
    got_k, got_v = _to_host(ko), _to_host(vo)
    del dk, dv, ko, vo, idx, code, eq
    torch.cuda.empty_cache()
    # element by element against the oracle (its output does not depend on p,
    # which its pins fix, so it runs one block per host core)
    cores = os.cpu_count() or 1
    wk, wv = oracle.sort(k, v, p=cores, threads=cores)
    assert np.array_equal(got_k, wk)
    assert np.array_equal(got_v, wv)


def test_2e28_int32_uniform_p2_full_compare(sorter):
    """The benchmark's workload: 2^28 uniform int32 keys, p = 2, in the
    benchmark's launch configuration (8192-key tiles).  Fast checks first
    (nondecreasing, two multiset hashes, sampled oracle ranks), then the whole
    output element by element against the oracle."""
    from paper_1105_6040_gb300.abi import Sorter
    n = 1 << 28
    x = W.uniform_int32(n, seed=W.DEFAULT_SEED)
    xt = _to_dev(x)
    s13 = Sorter(0, tile_log2=13)
    try:
        out = s13.sort_keys(xt, p=2)
        s13.sync()
    finally:
        s13.close()
    got = _to_host(out)
    del xt, out
    torch.cuda.empty_cache()
    assert np.all(got[1:] >= got[:-1])                      # nondecreasing
    cin, cout = oracle.encode(x), oracle.encode(got)
    assert oracle.multiset_hash(cin, 0) == oracle.multiset_hash(cout, 0)  # permutation
    assert oracle.multiset_hash(cin, 1) == oracle.multiset_hash(cout, 1)
    rng = np.random.default_rng(0)
    for k in np.concatenate([[0, n - 1, n // 2], rng.integers(0, n, 13)]):
        lt, le = oracle.rank_bounds(cin, int(cout[k]))
        assert lt <= k < le, k
    del cin, cout
    # element by element against the oracle (one block per host core: its
    # output does not depend on p, which its pins fix)
    cores = os.cpu_count() or 1
    want, _ = oracle.sort(x, p=cores, threads=cores)
    assert np.array_equal(got, want)


# ------------------------------------------------------------------ merge kernels

@pytest.mark.parametrize("merge_kernel,merge_vt,tile_log2,merge_tile_log2,consumer", [
    ("simple", 0, 12, 0, 0), ("tma", 16, 12, 0, 0), ("tma", 8, 12, 0, 0), ("tma", 16, 12, 11, 0),
    ("tma", 8, 12, 11, 0), ("tma", 16, 13, 11, 0), ("tma", 16, 13, 12, 0), ("auto", 0, 11, 11, 0),
    ("tma", 16, 12, 0, 1), ("tma", 8, 13, 12, 1), ("tma", 32, 12, 0, 0), ("tma", 32, 13, 0, 0),
    ("tma", 32, 12, 11, 1), ("tma", 32, 13, 13, 1)])
def test_merge_kernel_variants(merge_kernel, merge_vt, tile_log2, merge_tile_log2, consumer):
    """Every merge-pass kernel, consumer and merge-tile shape gives the
    oracle's output on every key/value type, ragged sizes, several p and
    segmented inputs."""
    from paper_1105_6040_gb300.abi import Sorter
    s = Sorter(0, merge_kernel=merge_kernel, merge_vt=merge_vt, tile_log2=tile_log2,
               merge_tile_log2=merge_tile_log2, merge_consumer=consumer)
    try:
        for n, p in ((3 * T + 7, 1), (100003, 3), (1 << 18, 6), (262139, 64)):
            check_keys(s, W.uniform_int32(n, n + p), p)
            check_keys(s, W.uniform_uint64(n, n + p + 1), p)
            check_keys(s, W.normal_float32_edges(n, n + p + 2), p)
        for vmaker in (W.index_payload, lambda n: W.uniform_uint64(n, 9)):
            for kmaker in (lambda n: W.uniform_int32(n, 8) % 300, lambda n: W.zipf_uint64(n, 7)):
                n, p = 77777, 5
                k, v = kmaker(n), vmaker(n)
                ko, vo = s.sort_pairs(_to_dev(k), _to_dev(v), p=p)
                s.sync()
                wk, wv = oracle.sort(k, v, p=p)
                assert np.array_equal(_bits(_to_host(ko)), _bits(wk))
                assert np.array_equal(_bits(_to_host(vo)), _bits(wv))
        lens = W.loguniform_lengths(400, 1, 1 << 15, seed=77)
        off = W.offsets_from_lengths(lens)
        k = W.uniform_int32(int(off[-1]), seed=78)
        res = s.sort_segmented(_to_dev(k), torch.from_numpy(off).cuda())
        s.sync()
        assert np.array_equal(_to_host(res), oracle.sort_segmented(k, off)[0])
    finally:
        s.close()


@pytest.mark.parametrize("merge_vt,consumer", [(8, 1), (16, 1), (32, 1), (8, 0), (16, 0), (32, 0)])
def test_merge_stage_reuse_repeated(merge_vt, consumer):
    """Stress for the TMA pipeline's stage ring: many short segmented merges,
    run ten times; every run must equal the oracle.  A consumer read that is
    not ordered before the bulk copy refilling its stage corrupts keys here
    (fast consumers, a producer that refills at once)."""
    from paper_1105_6040_gb300.abi import Sorter
    s = Sorter(0, merge_kernel="tma", merge_vt=merge_vt, tile_log2=12, merge_consumer=consumer)
    try:
        lens = W.loguniform_lengths(400, 1, 1 << 15, seed=77)
        off = W.offsets_from_lengths(lens)
        k = W.uniform_int32(int(off[-1]), seed=78)
        want = oracle.sort_segmented(k, off)[0]
        dk, doff = _to_dev(k), torch.from_numpy(off).cuda()
        for _ in range(10):
            res = s.sort_segmented(dk, doff)
            s.sync()
            assert np.array_equal(_to_host(res), want)
    finally:
        s.close()


def test_unaligned_buffers_fall_back(sorter):
    """Buffers that are not 16-byte aligned still sort correctly."""
    x = W.uniform_int32(50001, 88)
    base = torch.zeros(50001 + 3, dtype=torch.int32, device="cuda")
    src = base[1:50002]
    src.copy_(torch.from_numpy(x))
    outb = torch.zeros(50001 + 3, dtype=torch.int32, device="cuda")
    out = outb[3:50004]
    from paper_1105_6040_gb300 import abi
    abi.bs_sort_keys(sorter.h, src.data_ptr(), out.data_ptr(), x.size, "int32", 3,
                     torch.cuda.current_stream().cuda_stream)
    sorter.sync()
    assert np.array_equal(out.cpu().numpy(), np.sort(x))


# ------------------------------------------------------------------ failure detection

@pytest.mark.parametrize("persistent", [2, 0])
def test_bounded_wait_runs_out_and_reports_timeout(persistent):
    """A stage that nothing fills: the merge's bounded waits run out (in the
    persistent merge, the other CTAs' waits on the pairs that CTA never
    finishes too), the call reports BS_ERR_TIMEOUT, and the same handle sorts
    correctly after."""
    from paper_1105_6040_gb300 import abi
    from paper_1105_6040_gb300.abi import Sorter
    s = Sorter(0, merge_kernel="tma")
    try:
        abi.bs_set_option(s.h, "merge_persistent", persistent)
        x = W.uniform_int32(1 << 16, seed=123)
        d = _to_dev(x)
        abi.bs_set_option(s.h, "wait_limit_ms", 100)
        abi.bs_set_option(s.h, "test_withhold", 1)
        s.sort_keys(d, p=1)
        assert abi.bs_sync_status(s.h) == abi.BS_ERR_TIMEOUT
        abi.bs_set_option(s.h, "test_withhold", 0)
        out = s.sort_keys(d, p=1)
        s.sync()
        assert np.array_equal(_to_host(out), np.sort(x))
    finally:
        s.close()


# ------------------------------------------------------------------ odd-even schedule (Fig. 1)

@pytest.mark.parametrize("n,p", [(4, 3), (10, 4), (5000, 3), (T * 5 + 3, 7), (100003, 16),
                                 (1 << 18, 64), (300, 300), (77, 2)])
def test_oddeven_schedule_matches_oracle(n, p):
    from paper_1105_6040_gb300 import abi
    from paper_1105_6040_gb300.abi import Sorter
    s = Sorter(0)
    try:
        abi.bs_set_option(s.h, "merge_schedule", "oddeven")
        for x in (W.uniform_int32(n, n + p) % 1000, W.reverse_int32(n),
                  W.normal_float32_edges(n, 5)):
            got = gpu_keys(s, x, p)
            want, _ = oracle.sort(x, p=p, form="oddeven")
            assert np.array_equal(_bits(got), _bits(want)), (n, p)
        s.stats(reset=True)
        s.sort_keys(_to_dev(W.uniform_int32(n, 1)), p=p)
        counts, _ = s.stats(reset=True)
        lv = max(0, int(np.ceil(np.log2(max(1, -(-n // p) / T))))) if -(-n // p) > T else 0
        assert counts["merge"] == p + lv  # in-block levels, then exactly p compare-split rounds
    finally:
        s.close()


# ------------------------------------------------------------------ local sorts of Figs. 2 and 4

@pytest.mark.parametrize("local", ["quick", "bubble"])
def test_local_sort_many_tiles_per_cta(local):
    """Thousands of tiles, so every CTA of the persistent tile-sort grid runs
    many tiles back to back (quick sort's segment stack is shared state
    between tiles and rounds)."""
    from paper_1105_6040_gb300 import abi
    from paper_1105_6040_gb300.abi import Sorter
    s = Sorter(0)
    try:
        abi.bs_set_option(s.h, "local_sort", local)
        n = (1 << 22) if local == "quick" else (1 << 20)
        for x in (W.uniform_int32(n, 97), W.dup16_int32(n, 98)):
            got = gpu_keys(s, x, 2)
            assert np.array_equal(got, oracle.sort(x, p=2)[0]), (local, x[:4])
    finally:
        s.close()


@pytest.mark.parametrize("local", ["bubble", "quick"])
def test_local_sort_variants_match_oracle(local):
    from paper_1105_6040_gb300 import abi
    from paper_1105_6040_gb300.abi import Sorter
    s = Sorter(0)
    try:
        abi.bs_set_option(s.h, "local_sort", local)
        cases = [(W.uniform_int32(1, 1), 1), (W.uniform_int32(T + 5, 2), 1),
                 (W.uniform_int32(3 * T - 1, 3), 3), (W.dup16_int32(2 * T + 7, 4), 2),
                 (W.reverse_int32(T), 1), (W.sorted_int32(5000), 2),
                 (W.normal_float32_edges(20001, 5), 4), (W.uniform_uint64(9000, 6), 2)]
        for x, p in cases:
            got = gpu_keys(s, x, p)
            want, _ = oracle.sort(x, p=p, local=local if x.size <= 9000 else "merge")
            assert np.array_equal(_bits(got), _bits(want)), (local, x.dtype, x.size, p)
        lens = np.array([0, 1, 33, 4096, 5000, 2], dtype=np.int64)
        off = W.offsets_from_lengths(lens)
        k = W.uniform_int32(int(off[-1]), 7) % 50
        res = s.sort_segmented(_to_dev(k), torch.from_numpy(off).cuda())
        s.sync()
        assert np.array_equal(_to_host(res), oracle.sort_segmented(k, off)[0])
        # pair sorts ignore the option and stay stable
        kk, vv = W.uniform_uint64(7000, 8) % np.uint64(9), W.index_payload(7000)
        ko, vo = s.sort_pairs(_to_dev(kk), _to_dev(vv), p=2)
        s.sync()
        wk, wv = oracle.sort(kk, vv, p=2)
        assert np.array_equal(_to_host(ko), wk) and np.array_equal(_to_host(vo), wv)
    finally:
        s.close()
