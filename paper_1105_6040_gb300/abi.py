"""Thin Python binding of the C ABI in include/bsort.h (argument marshalling only).

Every ``bs_*`` function here forwards to the function of the same name in
``libbsort.so``; all sorting work runs in that library's CUDA kernels.  There is
no CPU fallback: if the library cannot be loaded, or a call fails, an exception
is raised.

``Sorter`` wraps a handle and takes torch tensors (torch supplies device memory
and streams only).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

BS_OK = 0
BS_ERR_INVALID_ARG = 1
BS_ERR_UNSUPPORTED_DTYPE = 2
BS_ERR_OUT_OF_MEMORY = 3
BS_ERR_CUDA = 4
BS_ERR_TIMEOUT = 5
BS_ERR_TOO_LARGE = 6

DTYPES = {"none": -1, "int32": 0, "uint32": 1, "float32": 2, "int64": 3, "uint64": 4, "float64": 5}
KERNEL_CLASSES = ("tile_sort", "merge", "partition", "setup")

# every entry point include/bsort.h declares: name -> (argtypes, restype)
_P, _I64, _INT = C.c_void_p, C.c_int64, C.c_int
SIGNATURES = {
    "bs_create": ([C.POINTER(C.c_void_p), _INT], _INT),
    "bs_destroy": ([_P], _INT),
    "bs_sort_keys": ([_P, _P, _P, _I64, _INT, _I64, _P], _INT),
    "bs_sort_pairs": ([_P, _P, _P, _P, _P, _I64, _INT, _INT, _I64, _P], _INT),
    "bs_sort_segmented": ([_P, _P, _P, _P, _P, _I64, _P, _I64, _I64, _INT, _INT, _P], _INT),
    "bs_sort_keys_host": ([_P, _P, _P, _I64, _INT, _I64], _INT),
    "bs_sort_keys_host_async": ([_P, _P, _P, _I64, _INT, _I64, _P], _INT),
    "bs_merge_runs": ([_P, _P, _P, _P, _P, _I64, _P, _I64, _INT, _INT, _P], _INT),
    "bs_sort_segmented_gather": ([_P, _P, _I64, _P, _P, _P, _P, _I64, _P, _I64, _I64, _INT, _INT,
                                  _P], _INT),
    "bs_workspace_bytes": ([_I64, _I64, _INT, _INT, C.POINTER(C.c_size_t)], _INT),
    "bs_reserve_workspace": ([_P, _I64, _I64, _INT, _INT, C.POINTER(C.c_size_t)], _INT),
    "bs_order_keys": ([_P, _P, _I64, _INT, _P], _INT),
    "bs_check_keys": ([_P, _I64, _INT, _P, _I64, _P, _INT, _P, _P], _INT),
    "bs_sync_status": ([_P], _INT),
    "bs_status_str": ([_INT], C.c_char_p),
    "bs_launch_stats": ([_P, C.POINTER(C.c_int64), C.POINTER(C.c_double), _INT], _INT),
    "bs_set_kernel_timing": ([_P, _INT], _INT),
    "bs_kernel_times": ([_P, C.POINTER(C.c_double), C.POINTER(C.c_int64)], _INT),
    "bs_set_tile_log2": ([_P, _INT], _INT),
    "bs_set_option": ([_P, _INT, _I64], _INT),
    "bs_sort_keys_noalloc": ([_P, _P, _I64, _INT, _I64, _P], _INT),
    "bs_graph_capture_segmented": ([_P, _P, _P, _P, _P, _I64, _P, _I64, _I64, _INT, _INT,
                                    C.POINTER(C.c_void_p)], _INT),
    "bs_graph_capture_keys": ([_P, _P, _P, _I64, _INT, _I64, C.POINTER(C.c_void_p)], _INT),
    "bs_graph_launch": ([_P, _P], _INT),
    "bs_graph_sync_status": ([_P], _INT),
    "bs_graph_destroy": ([_P], _INT),
}

_lib = None
_lock = threading.Lock()


class BsError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_str(status)} ({status})")


def load(build_if_missing: bool = True) -> C.CDLL:
    """Load libbsort.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.lib_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libbsort.so not found at {path}; run the build first")
            lib = C.CDLL(path)
            for name, (args, res) in SIGNATURES.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def status_str(status: int) -> str:
    return load().bs_status_str(int(status)).decode()


def _check(status: int, where: str) -> None:
    if status != BS_OK:
        raise BsError(status, where)


def dtype_code(dt) -> int:
    """bs_dtype code of a dtype name, numpy dtype or torch dtype."""
    if isinstance(dt, int):
        return dt
    name = str(dt).replace("torch.", "")
    if name not in DTYPES:
        raise BsError(BS_ERR_UNSUPPORTED_DTYPE, f"dtype {dt}")
    return DTYPES[name]


# ---------------------------------------------------------------- raw entry points


def bs_create(device: int = 0) -> int:
    h = C.c_void_p()
    _check(load().bs_create(C.byref(h), int(device)), "bs_create")
    return h.value


def bs_destroy(h: int) -> None:
    _check(load().bs_destroy(h), "bs_destroy")


def bs_sort_keys(h, d_in, d_out, n, kt, p, stream=0) -> None:
    _check(load().bs_sort_keys(h, d_in, d_out, int(n), dtype_code(kt), int(p), stream or None),
           "bs_sort_keys")


def bs_sort_pairs(h, d_kin, d_kout, d_vin, d_vout, n, kt, vt, p, stream=0) -> None:
    _check(load().bs_sort_pairs(h, d_kin, d_kout, d_vin, d_vout, int(n), dtype_code(kt),
                                dtype_code(vt), int(p), stream or None), "bs_sort_pairs")


def bs_sort_segmented(h, d_kin, d_kout, d_vin, d_vout, n, d_offsets, S, max_seg_len, kt, vt,
                      stream=0) -> None:
    _check(load().bs_sort_segmented(h, d_kin, d_kout, d_vin, d_vout, int(n), d_offsets, int(S),
                                    int(max_seg_len), dtype_code(kt), dtype_code(vt),
                                    stream or None), "bs_sort_segmented")


def bs_sort_segmented_gather(h, d_kin, n_in, d_src_offsets, d_kout, d_vin, d_vout, n, d_offsets,
                             S, max_seg_len, kt, vt, stream=0) -> None:
    _check(load().bs_sort_segmented_gather(h, d_kin, int(n_in), d_src_offsets, d_kout, d_vin,
                                           d_vout, int(n), d_offsets, int(S), int(max_seg_len),
                                           dtype_code(kt), dtype_code(vt), stream or None),
           "bs_sort_segmented_gather")


def bs_merge_runs(h, d_kin, d_kout, d_vin, d_vout, n, h_run_offsets, runs, kt, vt="none",
                  stream=0) -> None:
    import numpy as np
    off = np.ascontiguousarray(h_run_offsets, dtype=np.int64)
    _check(load().bs_merge_runs(h, d_kin, d_kout, d_vin, d_vout, int(n), off.ctypes.data,
                                int(runs), dtype_code(kt), dtype_code(vt), stream or None),
           "bs_merge_runs")


def bs_sort_keys_host(h, h_in, h_out, n, kt, p) -> None:
    _check(load().bs_sort_keys_host(h, h_in, h_out, int(n), dtype_code(kt), int(p)),
           "bs_sort_keys_host")


def bs_sort_keys_host_async(h, h_in, h_out, n, kt, p, stream=0) -> None:
    _check(load().bs_sort_keys_host_async(h, h_in, h_out, int(n), dtype_code(kt), int(p),
                                          stream or None), "bs_sort_keys_host_async")


def bs_workspace_bytes(n, S, kt, vt="none") -> int:
    out = C.c_size_t()
    _check(load().bs_workspace_bytes(int(n), int(S), dtype_code(kt), dtype_code(vt), C.byref(out)),
           "bs_workspace_bytes")
    return out.value


def bs_reserve_workspace(h, n, S, kt, vt="none") -> int:
    """Grow the handle's scratch now for a sort of n keys in S blocks or
    segments; returns the handle's scratch bytes."""
    out = C.c_size_t()
    _check(load().bs_reserve_workspace(h, int(n), int(S), dtype_code(kt), dtype_code(vt), C.byref(out)),
           "bs_reserve_workspace")
    return out.value


def bs_order_keys(d_in, d_out, n, kt, stream=0) -> None:
    """d_out (int64) <- keys' order-preserving codes as signed 64-bit integers."""
    _check(load().bs_order_keys(d_in, d_out, int(n), dtype_code(kt), stream or None), "bs_order_keys")


def order_keys(keys, stream=None):
    """A torch int64 tensor whose order (signed) is the library's sort order of
    `keys` (a CUDA tensor of a key dtype)."""
    import torch
    if not keys.is_cuda or not keys.is_contiguous():
        raise ValueError("keys must be a contiguous CUDA tensor")
    out = torch.empty(keys.numel(), dtype=torch.int64, device=keys.device)
    bs_order_keys(keys.data_ptr(), out.data_ptr(), keys.numel(), keys.dtype,
                  _stream_ptr(stream, keys.device))
    return out


class CheckResult(C.Structure):
    """bs_check_result: first offending positions (-1 = none) and the two
    multiset hashes of the keys' codes."""
    _fields_ = [("first_unsorted", C.c_int64), ("first_unstable", C.c_int64),
                ("hash_a", C.c_uint64), ("hash_b", C.c_uint64)]


def bs_check_keys(d_keys, n, kt, d_offsets=None, S=0, d_idx=None, it="none", stream=0) -> dict:
    """The device checkers (one pass): first_unsorted / first_unstable
    (-1 = none; segment starts excused when offsets are given) and hash_a /
    hash_b of the keys' codes.  Waits for the result."""
    r = CheckResult()
    _check(load().bs_check_keys(d_keys, int(n), dtype_code(kt), d_offsets, int(S), d_idx,
                                dtype_code(it) if d_idx else -1, C.byref(r), stream or None),
           "bs_check_keys")
    return {"first_unsorted": r.first_unsorted, "first_unstable": r.first_unstable,
            "hash_a": r.hash_a, "hash_b": r.hash_b}


def check_keys(keys, offsets=None, idx=None, stream=None) -> dict:
    """bs_check_keys on CUDA tensors (keys of a key dtype; offsets int64,
    S+1 entries; idx an integer tensor of payload positions)."""
    for t, name in ((keys, "keys"), (offsets, "offsets"), (idx, "idx")):
        if t is not None and (not t.is_cuda or not t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous CUDA tensor")
    return bs_check_keys(keys.data_ptr(), keys.numel(), keys.dtype,
                         None if offsets is None else offsets.data_ptr(),
                         0 if offsets is None else offsets.numel() - 1,
                         None if idx is None else idx.data_ptr(),
                         "none" if idx is None else idx.dtype, _stream_ptr(stream, keys.device))


def bs_sync_status(h) -> int:
    return int(load().bs_sync_status(h))


def bs_launch_stats(h, reset: bool = False, with_bytes: bool = True):
    counts = (C.c_int64 * 4)()
    byts = (C.c_double * 4)()
    _check(load().bs_launch_stats(h, counts, byts if with_bytes else None, int(reset)),
           "bs_launch_stats")
    return ({k: counts[i] for i, k in enumerate(KERNEL_CLASSES)},
            {k: byts[i] for i, k in enumerate(KERNEL_CLASSES)})


def bs_set_kernel_timing(h, enable: bool) -> None:
    _check(load().bs_set_kernel_timing(h, int(bool(enable))), "bs_set_kernel_timing")


def bs_kernel_times(h):
    ms = (C.c_double * 4)()
    n = (C.c_int64 * 4)()
    _check(load().bs_kernel_times(h, ms, n), "bs_kernel_times")
    return ({k: ms[i] for i, k in enumerate(KERNEL_CLASSES)},
            {k: n[i] for i, k in enumerate(KERNEL_CLASSES)})


def bs_set_tile_log2(h, tile_log2: int) -> None:
    _check(load().bs_set_tile_log2(h, int(tile_log2)), "bs_set_tile_log2")


OPTIONS = {"tile_log2": 0, "merge_kernel": 1, "merge_vt": 2, "wait_limit_ms": 3,
           "test_withhold": 4, "merge_schedule": 5, "local_sort": 6, "merge_tile_log2": 7,
           "merge_consumer": 8, "host_direct": 9, "count_bytes": 10,
           "merge_persistent": 11, "length_classes": 12, "host_slots": 13}
SCHEDULES = {"tree": 0, "oddeven": 1}
LOCAL_SORTS = {"merge": 0, "bubble": 1, "quick": 2}
MERGE_KERNELS = {"auto": 0, "simple": 1, "tma": 2}


def bs_set_option(h, option, value) -> None:
    if isinstance(option, str):
        option = OPTIONS[option]
    if isinstance(value, str):
        value = {OPTIONS["merge_schedule"]: SCHEDULES,
                 OPTIONS["local_sort"]: LOCAL_SORTS}.get(option, MERGE_KERNELS)[value]
    _check(load().bs_set_option(h, int(option), int(value)), "bs_set_option")


def bs_sort_keys_noalloc(d_in, d_out, n, kt, p, stream=0) -> None:
    """Key sort for callers that must not allocate GPU memory while sorting:
    the library's fixed scratch array is used instead of a handle's memory
    (at most 4 MiB of keys, p <= 1024; larger requests raise BS_ERR_TOO_LARGE).
    Calls share that array, so calls overlapping on the GPU must be avoided."""
    _check(load().bs_sort_keys_noalloc(d_in, d_out, int(n), dtype_code(kt), int(p), stream or None),
           "bs_sort_keys_noalloc")


def bs_graph_capture_segmented(h, d_kin, d_kout, d_vin, d_vout, n, d_offsets, S, max_seg_len,
                               kt, vt) -> int:
    g = C.c_void_p()
    _check(load().bs_graph_capture_segmented(h, d_kin, d_kout, d_vin, d_vout, int(n), d_offsets,
                                             int(S), int(max_seg_len), dtype_code(kt),
                                             dtype_code(vt), C.byref(g)),
           "bs_graph_capture_segmented")
    return g.value


def bs_graph_capture_keys(h, d_in, d_out, n, kt, p) -> int:
    g = C.c_void_p()
    _check(load().bs_graph_capture_keys(h, d_in, d_out, int(n), dtype_code(kt), int(p),
                                        C.byref(g)), "bs_graph_capture_keys")
    return g.value


def bs_graph_launch(g, stream=0) -> None:
    _check(load().bs_graph_launch(g, stream or None), "bs_graph_launch")


def bs_graph_sync_status(g) -> int:
    return int(load().bs_graph_sync_status(g))


def bs_graph_destroy(g) -> None:
    _check(load().bs_graph_destroy(g), "bs_graph_destroy")


class SortGraph:
    """A captured sort (bs_graph_*): replay with launch(), free with close()."""

    def __init__(self, g: int, keep=()):
        self.g = g
        self._keep = keep  # tensors the graph refers to

    def launch(self, stream=None):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        bs_graph_launch(self.g, int(s.cuda_stream))

    def sync(self):
        _check(bs_graph_sync_status(self.g), "bs_graph_sync_status")

    def close(self):
        if getattr(self, "g", None):
            bs_graph_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- torch front end


def _stream_ptr(stream, device) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return int(s.cuda_stream)


class Sorter:
    """A library handle on one CUDA device, taking torch tensors."""

    def __init__(self, device=None, tile_log2: int = 0, merge_kernel: str = "auto",
                 merge_vt: int = 0, merge_tile_log2: int = 0, merge_consumer: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Sorter needs a CUDA device; there is no CPU path")
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        self.h = bs_create(self.device.index)
        if tile_log2:
            bs_set_tile_log2(self.h, tile_log2)
        if merge_kernel != "auto":
            bs_set_option(self.h, "merge_kernel", merge_kernel)
        if merge_vt:
            bs_set_option(self.h, "merge_vt", merge_vt)
        if merge_tile_log2:
            bs_set_option(self.h, "merge_tile_log2", merge_tile_log2)
        if merge_consumer:
            bs_set_option(self.h, "merge_consumer", merge_consumer)

    def close(self):
        if getattr(self, "h", None):
            bs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_tensor(self, t, name):
        if not t.is_cuda or t.device != self.device or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous tensor on {self.device}")

    def sort_keys(self, keys, out=None, p: int = 1, stream=None):
        import torch
        self._check_tensor(keys, "keys")
        if out is None:
            out = torch.empty_like(keys)
        self._check_tensor(out, "out")
        bs_sort_keys(self.h, keys.data_ptr(), out.data_ptr(), keys.numel(), keys.dtype, p,
                     _stream_ptr(stream, self.device))
        return out

    def sort_pairs(self, keys, vals, kout=None, vout=None, p: int = 1, stream=None):
        import torch
        self._check_tensor(keys, "keys")
        self._check_tensor(vals, "vals")
        if vals.numel() != keys.numel():
            raise ValueError("keys and vals differ in length")
        kout = torch.empty_like(keys) if kout is None else kout
        vout = torch.empty_like(vals) if vout is None else vout
        bs_sort_pairs(self.h, keys.data_ptr(), kout.data_ptr(), vals.data_ptr(), vout.data_ptr(),
                      keys.numel(), keys.dtype, vals.dtype, p, _stream_ptr(stream, self.device))
        return kout, vout

    def sort_segmented(self, keys, offsets, vals=None, kout=None, vout=None,
                       max_seg_len: int = 0, stream=None):
        import torch
        self._check_tensor(keys, "keys")
        self._check_tensor(offsets, "offsets")
        if offsets.dtype != torch.int64:
            raise ValueError("offsets must be int64")
        kout = torch.empty_like(keys) if kout is None else kout
        if vals is not None:
            self._check_tensor(vals, "vals")
            vout = torch.empty_like(vals) if vout is None else vout
        bs_sort_segmented(self.h, keys.data_ptr(), kout.data_ptr(),
                          None if vals is None else vals.data_ptr(),
                          None if vals is None else vout.data_ptr(),
                          keys.numel(), offsets.data_ptr(), offsets.numel() - 1, max_seg_len,
                          keys.dtype, "none" if vals is None else vals.dtype,
                          _stream_ptr(stream, self.device))
        return (kout, vout) if vals is not None else kout

    def sort_gathered(self, pool, src_offsets, offsets, kout=None, max_seg_len: int = 0,
                      stream=None):
        """Sort S segments whose keys sit at src_offsets[s] of `pool` into
        kout[offsets[s] : offsets[s+1]] in one call (keys only)."""
        import torch
        for t, name in ((pool, "pool"), (src_offsets, "src_offsets"), (offsets, "offsets")):
            self._check_tensor(t, name)
        n = int(offsets[-1].item()) if kout is None else kout.numel()
        kout = torch.empty(n, dtype=pool.dtype, device=pool.device) if kout is None else kout
        bs_sort_segmented_gather(self.h, pool.data_ptr(), pool.numel(), src_offsets.data_ptr(),
                                 kout.data_ptr(), None, None, kout.numel(), offsets.data_ptr(),
                                 offsets.numel() - 1, max_seg_len, pool.dtype, "none",
                                 _stream_ptr(stream, self.device))
        return kout

    def capture_segmented(self, keys, offsets, kout, vals=None, vout=None, max_seg_len: int = 0):
        """Capture bs_sort_segmented on these tensors into a replayable graph."""
        for t, name in ((keys, "keys"), (offsets, "offsets"), (kout, "kout")):
            self._check_tensor(t, name)
        g = bs_graph_capture_segmented(
            self.h, keys.data_ptr(), kout.data_ptr(),
            None if vals is None else vals.data_ptr(), None if vals is None else vout.data_ptr(),
            keys.numel(), offsets.data_ptr(), offsets.numel() - 1, max_seg_len, keys.dtype,
            "none" if vals is None else vals.dtype)
        return SortGraph(g, keep=(keys, offsets, kout, vals, vout))

    def capture_keys(self, keys, out, p: int = 1):
        self._check_tensor(keys, "keys")
        self._check_tensor(out, "out")
        g = bs_graph_capture_keys(self.h, keys.data_ptr(), out.data_ptr(), keys.numel(),
                                  keys.dtype, p)
        return SortGraph(g, keep=(keys, out))

    def merge_runs(self, keys, run_offsets, out=None, stream=None):
        """Merge sorted runs keys[run_offsets[r]:run_offsets[r+1]] into one
        sorted tensor (run_offsets: host sequence of runs+1 ints)."""
        import torch
        self._check_tensor(keys, "keys")
        out = torch.empty_like(keys) if out is None else out
        bs_merge_runs(self.h, keys.data_ptr(), out.data_ptr(), None, None, keys.numel(),
                      run_offsets, len(run_offsets) - 1, keys.dtype, "none",
                      _stream_ptr(stream, self.device))
        return out

    def sort_keys_host(self, h_in, h_out=None, p: int = 1):
        """Sort a host (CPU) tensor through the library's host-buffer entry point."""
        import torch
        if h_in.is_cuda or not h_in.is_contiguous():
            raise ValueError("h_in must be a contiguous CPU tensor")
        h_out = torch.empty_like(h_in) if h_out is None else h_out
        bs_sort_keys_host(self.h, h_in.data_ptr(), h_out.data_ptr(), h_in.numel(), h_in.dtype, p)
        return h_out

    def sort_keys_host_async(self, h_in, h_out, p: int = 1, stream=None):
        """Enqueue a sort of host tensor h_in into host tensor h_out (copy in,
        sort on `stream`, copy out) and return at once; successive calls
        overlap their copies with each other's sorts.  The results are
        complete after sync().  Use page-locked tensors."""
        for t, name in ((h_in, "h_in"), (h_out, "h_out")):
            if t.is_cuda or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous CPU tensor")
        if h_out.numel() != h_in.numel() or h_out.dtype != h_in.dtype:
            raise ValueError("h_out must match h_in in size and dtype")
        bs_sort_keys_host_async(self.h, h_in.data_ptr(), h_out.data_ptr(), h_in.numel(), h_in.dtype, p,
                                _stream_ptr(stream, self.device))
        return h_out

    def sync(self) -> None:
        _check(bs_sync_status(self.h), "bs_sync_status")

    def stats(self, reset: bool = False):
        return bs_launch_stats(self.h, reset=reset)

    def set_timing(self, enable: bool) -> None:
        bs_set_kernel_timing(self.h, enable)

    def kernel_times(self):
        return bs_kernel_times(self.h)
