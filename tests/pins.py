"""Pins of the CPU oracle: facts fixed by the definition of sorting and by the
IEEE 754 total order, checked without trusting the oracle itself.

Each pin takes a loaded oracle build and raises AssertionError on a mismatch.
``run_pins`` runs them all and returns the names of those that failed; the
mutation tests use it to show that every planted mistake is caught.

What pins what:
* codec_*: known codes of integer extremes, the IEEE 754-2008 totalOrder lists
  in tests/golden/ (Sec. 5.10), numpy's comparisons on random values, and the
  decode(encode(x)) round trip bit for bit.
* brute_*: every permutation of small multisets (n <= 8) must give the one
  sorted list, and -- with payload = input position -- the payload order of a
  stable sort (equal codes in input order), for every local sort / merge form.
* closed forms: sorted input maps to itself, reverse input to its reversal,
  the 16-distinct input to 16 constant runs with the generator's histogram.
* library special case: numpy's stable sort / argsort on the same codes.
* p-invariance: every block count and merge form gives the same output
  (the method's result does not depend on the decomposition).
* segmented: each segment equals numpy's sort of that segment.
* checkers: rank bounds against numpy counts, hash sensitivity.
"""
from __future__ import annotations

import itertools
import os

import numpy as np

from paper_1105_6040_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden_words(name: str) -> list[int]:
    words = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            words.append(int(line.split()[0], 16))
    return words


# --------------------------------------------------------------------------- codec

def pin_codec_integer_extremes(orc):
    i32 = np.array([-2**31, -1, 0, 1, 2**31 - 1], dtype=np.int32)
    assert orc.encode(i32).tolist() == [0, 0x7FFFFFFF, 0x80000000, 0x80000001, 0xFFFFFFFF]
    u32 = np.array([0, 1, 2**32 - 1], dtype=np.uint32)
    assert orc.encode(u32).tolist() == [0, 1, 2**32 - 1]
    i64 = np.array([-2**63, -1, 0, 2**63 - 1], dtype=np.int64)
    assert orc.encode(i64).tolist() == [0, 2**63 - 1, 2**63, 2**64 - 1]
    u64 = np.array([0, 2**64 - 1], dtype=np.uint64)
    assert orc.encode(u64).tolist() == [0, 2**64 - 1]


def pin_codec_float_total_order(orc):
    for fname, itype, ftype in (("float32_total_order.txt", np.uint32, np.float32),
                                ("float64_total_order.txt", np.uint64, np.float64)):
        words = np.array(_golden_words(fname), dtype=itype)
        codes = orc.encode(words.view(ftype))
        assert np.all(np.diff(codes.astype(object)) > 0), fname
        # sorting a shuffled copy gives back exactly the listed patterns
        rng = np.random.default_rng(7)
        shuffled = words[rng.permutation(words.size)].view(ftype)
        out, _ = orc.sort(shuffled, p=3)
        assert np.array_equal(out.view(itype), words), fname


def pin_codec_order_random(orc):
    rng = np.random.default_rng(11)
    for dt in (np.int32, np.int64):
        info = np.iinfo(dt)
        a = rng.integers(info.min, info.max, size=4000, dtype=dt, endpoint=True)
        b = rng.integers(info.min, info.max, size=4000, dtype=dt, endpoint=True)
        ca, cb = orc.encode(a), orc.encode(b)
        assert np.array_equal(a < b, ca < cb) and np.array_equal(a == b, ca == cb)
    for dt in (np.float32, np.float64):
        a = rng.standard_normal(4000).astype(dt) * dt(1e3)
        b = rng.standard_normal(4000).astype(dt) * dt(1e3)
        b[:100] = a[:100]
        ca, cb = orc.encode(a), orc.encode(b)
        assert np.array_equal(a < b, ca < cb) and np.array_equal(a == b, ca == cb)


def pin_codec_round_trip(orc):
    for keys in (W.uniform_int32(5000, 3), W.uniform_int32(5000, 4).view(np.uint32),
                 W.uniform_float32_bits(5000, 5), W.uniform_uint64(5000, 6),
                 W.uniform_uint64(5000, 7).view(np.int64), W.uniform_float64_bits(5000, 8)):
        back = orc.decode(orc.encode(keys), keys.dtype)
        iv = np.uint32 if keys.dtype.itemsize == 4 else np.uint64
        assert np.array_equal(back.view(iv), keys.view(iv)), keys.dtype


# --------------------------------------------------------------------------- brute force

def _perms(n: int) -> np.ndarray:
    return np.array(list(itertools.permutations(range(n))), dtype=np.int64)


def _brute(orc, base: list[int], configs, check_stable=True, every=1):
    base = np.array(base, dtype=np.uint64)
    n = base.size
    want_codes = np.array(sorted(base.tolist()), dtype=np.uint64)
    perms = _perms(n)[::every]
    pos = np.arange(n, dtype=np.uint64)
    for perm in perms:
        codes = base[perm]
        # stable order: by (code, input position) -- the definition of stability
        want_pay = np.array(sorted(range(n), key=lambda i: (int(codes[i]), i)), dtype=np.uint64)
        for (p, local, form) in configs:
            vals = None if local == "quick" else pos
            out, pay = orc.sort_codes(codes, vals, p=p, local=local, form=form)
            assert np.array_equal(out, want_codes), (base.tolist(), perm.tolist(), p, local, form)
            if check_stable and vals is not None:
                assert np.array_equal(pay, want_pay), ("unstable", perm.tolist(), p, local, form)


def pin_brute_n8(orc):
    cfgs = [(3, "merge", "tree"), (5, "merge", "oddeven"), (8, "merge", "gather")]
    _brute(orc, [3, 1, 3, 2, 1, 3, 0, 2], cfgs)                       # duplicates
    _brute(orc, [9, 2, 7, 4, 5, 0, 8, 1], [(3, "merge", "tree")], every=3)  # distinct
    _brute(orc, [4] * 8, [(4, "merge", "oddeven")], every=7)            # all equal


def pin_brute_n6_all_forms(orc):
    cfgs = [(p, local, form) for p in (1, 2, 3, 4, 6, 7)
            for local in ("merge", "bubble", "quick")
            for form in ("tree", "oddeven", "gather")]
    _brute(orc, [2, 0, 2, 1, 0, 2], cfgs)
    _brute(orc, [5, 3, 1, 4, 0, 2], cfgs[::5])


def pin_brute_float_specials(orc):
    f = np.array([np.inf, -np.inf, -0.0, 0.0, np.nan, -1.0, 1.0], dtype=np.float32)
    want = np.array(sorted(orc.encode(f).tolist()), dtype=np.uint64)
    for perm in _perms(7)[::11]:
        out, _ = orc.sort(f[perm], p=3)
        assert np.array_equal(orc.encode(out), want)
    # -0 sorts strictly before +0 and -inf/+inf bracket the finite values
    out, _ = orc.sort(f, p=2)
    bits = out.view(np.uint32)
    assert bits[0] == 0xFF800000 and bits[2] == 0x80000000 and bits[3] == 0 and bits[5] == 0x7F800000


# --------------------------------------------------------------------------- closed forms

def pin_closed_sorted_reverse(orc):
    n = 3000
    s = W.sorted_int32(n)
    assert np.all(np.diff(s.astype(np.int64)) > 0)
    for p in (1, 2, 7, 64):
        out, _ = orc.sort(s, p=p)
        assert np.array_equal(out, s)
        out, _ = orc.sort(W.reverse_int32(n), p=p)
        assert np.array_equal(out, s)
        out, _ = orc.sort(W.reverse_int32(n), p=p, form="oddeven")
        assert np.array_equal(out, s)


def pin_closed_dup16(orc):
    n = 5000
    x = W.dup16_int32(n, seed=21)
    vals, counts = np.unique(x, return_counts=True)
    assert vals.size == 16
    out, pay = orc.sort(x, W.index_payload(n), p=5)
    # 16 constant runs, in increasing value order, of the input's histogram
    expect = np.repeat(vals, counts)
    assert np.array_equal(out, expect)
    # inside each run the payload (= input index) increases: stability
    start = 0
    for c in counts:
        run = pay[start:start + c].astype(np.int64)
        assert np.all(np.diff(run) > 0)
        start += c


def pin_library_stable(orc):
    for n, seed, p in ((1, 1, 1), (2, 2, 2), (97, 3, 4), (4096, 4, 16), (7777, 5, 13)):
        x = W.uniform_int32(n, seed) % 50  # many ties
        idx = W.index_payload(n)
        out, pay = orc.sort(x, idx, p=p)
        assert np.array_equal(out, np.sort(x, kind="stable"))
        assert np.array_equal(pay, np.argsort(x, kind="stable").astype(np.int32))
    k = W.zipf_uint64(6000, seed=9)
    out, pay = orc.sort(k, W.index_payload(k.size), p=6, form="oddeven")
    assert np.array_equal(out, np.sort(k, kind="stable"))
    assert np.array_equal(pay, np.argsort(k, kind="stable").astype(np.int32))


def pin_p_invariance(orc):
    x = W.uniform_int32(1500, seed=31) % 200
    ref, _ = orc.sort(x, p=1)
    for p in (2, 3, 7, 64, 1499, 1500, 1501, 5000):
        for form in ("tree", "oddeven", "gather"):
            out, _ = orc.sort(x, p=p, form=form)
            assert np.array_equal(out, ref), (p, form)
    y = x[:300]
    ref_y, _ = orc.sort(y, p=1)
    for p in (1, 2, 5, 17):
        for local in ("bubble", "quick"):
            out, _ = orc.sort(y, p=p, local=local)
            assert np.array_equal(out, ref_y), (p, local)


def pin_bounds(orc):
    for n, p in ((10, 3), (0, 1), (7, 7), (2**28, 4096), (1000, 7)):
        b = orc.block_bounds(n, p)
        want = [(i * n) // p for i in range(p + 1)]
        assert b.tolist() == want
        sizes = np.diff(b)
        if n:
            assert sizes.max() - sizes.min() <= 1


def pin_segmented(orc):
    lens = np.array([0, 1, 5, 0, 33, 2, 100, 1], dtype=np.int64)
    off = W.offsets_from_lengths(lens)
    x = W.uniform_int32(int(off[-1]), seed=41) % 9
    out, pay = orc.sort_segmented(x, off, W.index_payload(x.size))
    for s in range(lens.size):
        a, b = off[s], off[s + 1]
        assert np.array_equal(out[a:b], np.sort(x[a:b], kind="stable"))
        assert np.array_equal(pay[a:b], a + np.argsort(x[a:b], kind="stable"))


def pin_checkers(orc):
    x = W.uniform_int32(2000, seed=51)
    c = orc.encode(x)
    assert not orc.is_nondecreasing(c) and orc.is_nondecreasing(np.sort(c))
    assert orc.multiset_hash(c, 0) == orc.multiset_hash(c[::-1], 0)
    assert orc.multiset_hash(c, 1) == orc.multiset_hash(np.sort(c), 1)
    d = c.copy()
    d[5] ^= np.uint64(1)
    assert orc.multiset_hash(d, 0) != orc.multiset_hash(c, 0)
    assert orc.multiset_hash(d, 1) != orc.multiset_hash(c, 1)
    for v in (int(c[0]), int(c[17]), 0, 2**32 - 1):
        lt, le = orc.rank_bounds(c, v)
        assert lt == int(np.sum(c < np.uint64(v))) and le == int(np.sum(c <= np.uint64(v)))


PINS = [
    pin_codec_integer_extremes, pin_codec_float_total_order, pin_codec_order_random,
    pin_codec_round_trip, pin_bounds, pin_closed_sorted_reverse, pin_closed_dup16,
    pin_library_stable, pin_p_invariance, pin_segmented, pin_checkers,
    pin_brute_float_specials, pin_brute_n6_all_forms, pin_brute_n8,
]


def run_pins(orc, stop_at_first: bool = False) -> list[str]:
    failed = []
    for pin in PINS:
        try:
            pin(orc)
        except AssertionError:
            failed.append(pin.__name__)
            if stop_at_first:
                break
    return failed
