"""ctypes front end of the CPU oracle (test infrastructure only).

Functions mirror the paper's scatter / sort / merge paradigm (El-Nashar 2011,
Sec. 3.2, Fig. 1) on numpy arrays:

* :func:`encode` / :func:`decode` -- order-preserving unsigned codes
  (integers: sign flip; floats: IEEE 754-2008 totalOrder bit patterns).
* :func:`sort` -- scatter into ``p`` blocks, sort each block with the chosen
  local sort (Fig. 3 merge, Fig. 2 bubble, Fig. 4 quick), merge the blocks with
  the chosen form (pairwise ``tree``, ``oddeven`` compare-split, ``gather``).
* :func:`sort_segmented` -- each segment sorted on its own (sort phase only).
* checkers: :func:`is_nondecreasing`, :func:`multiset_hash`,
  :func:`rank_bounds`.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

__all__ = [
    "OracleLib", "load", "encode", "decode", "sort", "sort_segmented",
    "is_nondecreasing", "multiset_hash", "rank_bounds", "block_bounds",
    "DTYPES", "LOCAL", "FORMS", "default_threads",
]

DTYPES = {"int32": 0, "uint32": 1, "float32": 2, "int64": 3, "uint64": 4, "float64": 5}
LOCAL = {"merge": 0, "bubble": 1, "quick": 2}
FORMS = {"tree": 0, "oddeven": 1, "gather": 2}

_P = C.c_void_p
_I64 = C.c_int64


class OracleLib:
    """One loaded build of the oracle (the default one, or a mutation variant)."""

    def __init__(self, path: str):
        self.path = path
        lib = C.CDLL(path)
        lib.orc_encode.argtypes = [_P, C.c_int, _I64, _P]
        lib.orc_decode.argtypes = [_P, C.c_int, _I64, _P]
        lib.orc_block_bounds.argtypes = [_I64, _I64, _P]
        lib.orc_sort_records.argtypes = [_P, _P, _I64, _I64, C.c_int, C.c_int, C.c_int]
        lib.orc_sort_segments.argtypes = [_P, _P, _P, _I64, C.c_int]
        lib.orc_is_nondecreasing.argtypes = [_P, _I64]
        lib.orc_multiset_hash.argtypes = [_P, _I64, C.c_int]
        lib.orc_multiset_hash.restype = C.c_uint64
        lib.orc_rank_bounds.argtypes = [_P, _I64, C.c_uint64, _P, _P]
        for f in ("orc_encode", "orc_decode", "orc_block_bounds", "orc_sort_records",
                  "orc_sort_segments", "orc_is_nondecreasing", "orc_rank_bounds"):
            getattr(lib, f).restype = C.c_int
        self.lib = lib

    # -- codec ------------------------------------------------------------
    def encode(self, keys: np.ndarray) -> np.ndarray:
        keys = np.ascontiguousarray(keys)
        dt = DTYPES[keys.dtype.name]
        codes = np.empty(keys.size, dtype=np.uint64)
        rc = self.lib.orc_encode(keys.ctypes.data, dt, keys.size, codes.ctypes.data)
        if rc:
            raise ValueError(f"orc_encode failed ({rc})")
        return codes

    def decode(self, codes: np.ndarray, dtype) -> np.ndarray:
        codes = np.ascontiguousarray(codes, dtype=np.uint64)
        out = np.empty(codes.size, dtype=np.dtype(dtype))
        rc = self.lib.orc_decode(codes.ctypes.data, DTYPES[out.dtype.name], codes.size,
                                 out.ctypes.data)
        if rc:
            raise ValueError(f"orc_decode failed ({rc})")
        return out

    def block_bounds(self, n: int, p: int) -> np.ndarray:
        b = np.empty(p + 1, dtype=np.int64)
        if self.lib.orc_block_bounds(n, p, b.ctypes.data):
            raise ValueError("bad n/p")
        return b

    # -- the method --------------------------------------------------------
    def sort_codes(self, codes: np.ndarray, vals: np.ndarray | None = None, p: int = 1,
                   local: str = "merge", form: str = "tree", threads: int = 1):
        codes = np.array(codes, dtype=np.uint64, copy=True)
        v = None if vals is None else np.array(vals, dtype=np.uint64, copy=True)
        rc = self.lib.orc_sort_records(codes.ctypes.data, None if v is None else v.ctypes.data,
                                       codes.size, int(p), LOCAL[local], FORMS[form],
                                       int(threads))
        if rc:
            raise ValueError(f"orc_sort_records failed ({rc})")
        return codes, v

    def sort(self, keys: np.ndarray, vals: np.ndarray | None = None, p: int = 1,
             local: str = "merge", form: str = "tree", threads: int = 1):
        """Sort keys (and carry vals) with the paper's paradigm; returns
        (sorted_keys, sorted_vals_or_None) in the input dtypes."""
        keys = np.ascontiguousarray(keys)
        codes = self.encode(keys)
        v64 = None
        if vals is not None:
            vals = np.ascontiguousarray(vals)
            v64 = _payload_to_u64(vals)
        codes, v64 = self.sort_codes(codes, v64, p=p, local=local, form=form, threads=threads)
        out_k = self.decode(codes, keys.dtype)
        out_v = None if vals is None else _u64_to_payload(v64, vals.dtype)
        return out_k, out_v

    def sort_segmented(self, keys: np.ndarray, offsets: np.ndarray,
                       vals: np.ndarray | None = None, threads: int = 1):
        keys = np.ascontiguousarray(keys)
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        codes = self.encode(keys)
        v64 = None if vals is None else _payload_to_u64(np.ascontiguousarray(vals))
        rc = self.lib.orc_sort_segments(codes.ctypes.data,
                                        None if v64 is None else v64.ctypes.data,
                                        off.ctypes.data, off.size - 1, int(threads))
        if rc:
            raise ValueError(f"orc_sort_segments failed ({rc})")
        out_k = self.decode(codes, keys.dtype)
        out_v = None if vals is None else _u64_to_payload(v64, vals.dtype)
        return out_k, out_v

    # -- checkers ----------------------------------------------------------
    def is_nondecreasing(self, codes: np.ndarray) -> bool:
        codes = np.ascontiguousarray(codes, dtype=np.uint64)
        return bool(self.lib.orc_is_nondecreasing(codes.ctypes.data, codes.size))

    def multiset_hash(self, codes: np.ndarray, which: int = 0) -> int:
        codes = np.ascontiguousarray(codes, dtype=np.uint64)
        return int(self.lib.orc_multiset_hash(codes.ctypes.data, codes.size, which))

    def rank_bounds(self, codes: np.ndarray, v: int):
        codes = np.ascontiguousarray(codes, dtype=np.uint64)
        lt, le = C.c_int64(), C.c_int64()
        self.lib.orc_rank_bounds(codes.ctypes.data, codes.size, C.c_uint64(int(v)),
                                 C.byref(lt), C.byref(le))
        return lt.value, le.value


def _payload_to_u64(vals: np.ndarray) -> np.ndarray:
    """Payload bits widened to uint64 (the oracle carries them unchanged)."""
    if vals.dtype.itemsize == 4:
        return vals.view(np.uint32).astype(np.uint64)
    if vals.dtype.itemsize == 8:
        return vals.view(np.uint64).copy()
    raise ValueError("payload must be 4 or 8 bytes wide")


def _u64_to_payload(v: np.ndarray, dtype) -> np.ndarray:
    dtype = np.dtype(dtype)
    if dtype.itemsize == 4:
        return v.astype(np.uint32).view(dtype)
    return v.view(dtype).copy()


_DEFAULT: OracleLib | None = None


def load(mutation: int = 0, out_dir: str | None = None) -> OracleLib:
    """Build if needed and load the oracle (mutation 0 = the real oracle)."""
    global _DEFAULT
    if mutation == 0 and out_dir is None:
        if _DEFAULT is None:
            _DEFAULT = OracleLib(_build.build())
        return _DEFAULT
    return OracleLib(_build.build(mutation=mutation, out_dir=out_dir))


def encode(keys):
    return load().encode(keys)


def decode(codes, dtype):
    return load().decode(codes, dtype)


def block_bounds(n, p):
    return load().block_bounds(n, p)


def sort(keys, vals=None, p=1, local="merge", form="tree", threads=1):
    return load().sort(keys, vals, p=p, local=local, form=form, threads=threads)


def sort_segmented(keys, offsets, vals=None, threads=1):
    return load().sort_segmented(keys, offsets, vals, threads=threads)


def is_nondecreasing(codes):
    return load().is_nondecreasing(codes)


def multiset_hash(codes, which=0):
    return load().multiset_hash(codes, which)


def rank_bounds(codes, v):
    return load().rank_bounds(codes, v)


def default_threads() -> int:
    return os.cpu_count() or 1
