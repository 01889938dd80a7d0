"""Autotuner for the sort's launch shapes.

The tunable knobs are the sort-phase tile size T = 2^tile_log2 keys (keys
alone: 128 or 256 threads per CTA with 32 keys each for 4096- and 8192-key
tiles, 128 threads with 16 keys for 2048; pairs: 128, 256 or 512 threads
with 16 pairs each), the merge-pass output tile
(the sort tile, or 4096 keys under 8192-key sort tiles), the merge-pass
kernel (the TMA pipeline or the plain shared-memory one) and, for the TMA
pipeline, the keys per consumer thread (the library's choice by item size:
32 for 32-bit keys alone, else 16; or 16 or 8 explicitly).  Results never
depend on them; speed does.

``tune(...)`` times every candidate on the caller's own inputs with CUDA
events (after a warm-up run), keeps the fastest, and remembers it in a JSON
cache keyed by the workload class: device name and SM count, call kind
(keys / pairs / segmented), key and value dtypes, log2 of the key count,
and for segmented calls log2 of the mean and maximum segment length.  The
cache lives in ``_build/autotune.json`` next to the library unless the
BS_AUTOTUNE_CACHE environment variable names another file.
"""
from __future__ import annotations

import json
import math
import os
import threading

from . import abi

TILE_LOG2 = (11, 12, 13)
MERGE_KERNELS = ("auto", "simple")
# (tile_log2, merge_tile_log2 (0: the sort tile), merge_kernel, merge_vt (0: by item size))
CANDIDATES = [(t, 0, "auto", 0) for t in TILE_LOG2] + [(13, 12, "auto", 0)] + \
    [(t, 0, "auto", 16) for t in (11, 12)] + [(t, 0, "auto", 8) for t in (11, 12)] + \
    [(t, 0, "simple", 16) for t in (11, 12)]

_lock = threading.Lock()


def cache_path() -> str:
    env = os.environ.get("BS_AUTOTUNE_CACHE")
    if env:
        return env
    from . import build
    return os.path.join(build.OUT_DIR, "autotune.json")


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(cache: dict) -> None:
    path = cache_path()
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _bucket(x: float) -> int:
    return int(round(math.log2(max(1.0, float(x)))))


def workload_key(kind: str, keys, vals=None, offsets=None, max_seg_len: int = 0) -> str:
    import torch
    dev = torch.cuda.get_device_properties(keys.device)
    parts = [dev.name.replace(" ", "_"), f"sm{dev.multi_processor_count}", kind,
             str(keys.dtype).replace("torch.", ""),
             "none" if vals is None else str(vals.dtype).replace("torch.", ""),
             f"n{_bucket(keys.numel())}"]
    if offsets is not None:
        S = max(1, offsets.numel() - 1)
        parts.append(f"mean{_bucket(keys.numel() / S)}")
        parts.append(f"max{_bucket(max_seg_len or keys.numel())}")
    return "|".join(parts)


def lookup(key: str):
    with _lock:
        return _load().get(key)


def apply(sorter: abi.Sorter, cfg: dict) -> None:
    abi.bs_set_option(sorter.h, "tile_log2", cfg["tile_log2"])
    abi.bs_set_option(sorter.h, "merge_tile_log2", cfg.get("merge_tile_log2", 0))
    abi.bs_set_option(sorter.h, "merge_kernel", cfg["merge_kernel"])
    abi.bs_set_option(sorter.h, "merge_vt", cfg.get("merge_vt", 0))


def _time_call(fn, repeats: int) -> float:
    import torch
    fn()  # warm-up (also grows the workspace)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune(sorter: abi.Sorter, kind: str, keys, vals=None, offsets=None, p: int = 1,
         max_seg_len: int = 0, repeats: int = 2, force: bool = False) -> dict:
    """Pick the launch shape for this workload class, apply it to
    `sorter` and return it.  kind: "keys", "pairs" or "segmented"."""
    import torch
    key = workload_key(kind, keys, vals, offsets, max_seg_len)
    if not force:
        cfg = lookup(key)
        if cfg:
            apply(sorter, cfg)
            return cfg
    kout = torch.empty_like(keys)
    vout = None if vals is None else torch.empty_like(vals)

    def run():
        if kind == "keys":
            sorter.sort_keys(keys, out=kout, p=p)
        elif kind == "pairs":
            sorter.sort_pairs(keys, vals, kout=kout, vout=vout, p=p)
        else:
            sorter.sort_segmented(keys, offsets, vals, kout=kout, vout=vout, max_seg_len=max_seg_len)

    timings = {}
    for tile, mtile, merge, vt in CANDIDATES:
        apply(sorter, {"tile_log2": tile, "merge_tile_log2": mtile, "merge_kernel": merge, "merge_vt": vt})
        timings[f"{tile}/{mtile}/{merge}/{vt}"] = _time_call(run, repeats)
    sorter.sync()
    best = min(timings, key=timings.get)
    tile, mtile, merge, vt = best.split("/")
    cfg = {"tile_log2": int(tile), "merge_tile_log2": int(mtile), "merge_kernel": merge, "merge_vt": int(vt),
           "ms": timings[best], "timings_ms": timings}
    with _lock:
        cache = _load()
        cache[key] = cfg
        _store(cache)
    apply(sorter, cfg)
    return cfg
