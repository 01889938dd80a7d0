"""The C-ABI library builds, loads and exports every entry point include/bsort.h
declares; host-side argument checks answer without a GPU (CPU only)."""
import ctypes as C

import numpy as np
import os
import re

import pytest

from paper_1105_6040_gb300 import abi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "bsort.h")).read()
    return sorted(set(re.findall(r"^(?:bs_status|const char \*)\s*(bs_\w+)\(", src, re.M)))


def test_header_declares_the_boundary():
    names = declared_entry_points()
    for must in ("bs_create", "bs_destroy", "bs_sort_keys", "bs_sort_pairs", "bs_sort_segmented",
                 "bs_workspace_bytes", "bs_sync_status", "bs_status_str"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = abi.load()
    for name in declared_entry_points():
        assert hasattr(lib, name), name
        assert name in abi.SIGNATURES, f"binding lacks {name}"


def test_status_strings():
    assert abi.status_str(abi.BS_OK) == "BS_OK"
    assert abi.status_str(abi.BS_ERR_TIMEOUT) == "BS_ERR_TIMEOUT"
    assert abi.status_str(99) == "BS_ERR_UNKNOWN"


def test_null_handle_and_bad_args_rejected_synchronously():
    lib = abi.load()
    assert lib.bs_sort_keys(None, None, None, 10, 0, 1, None) == abi.BS_ERR_INVALID_ARG
    assert lib.bs_sort_pairs(None, None, None, None, None, 10, 0, 0, 1, None) == abi.BS_ERR_INVALID_ARG
    assert lib.bs_sort_segmented(None, None, None, None, None, 0, None, 0, 0, 0, -1, None) == \
        abi.BS_ERR_INVALID_ARG
    assert lib.bs_sync_status(None) == abi.BS_ERR_INVALID_ARG
    assert lib.bs_create(None, 0) == abi.BS_ERR_INVALID_ARG
    assert lib.bs_destroy(None) == abi.BS_OK
    assert lib.bs_set_tile_log2(None, 12) == abi.BS_ERR_INVALID_ARG


def test_workspace_bytes_is_host_only_and_grows_with_n():
    a = abi.bs_workspace_bytes(1 << 20, 2, "int32")
    b = abi.bs_workspace_bytes(1 << 22, 2, "int32")
    c = abi.bs_workspace_bytes(1 << 20, 2, "uint64", "int32")
    assert (1 << 22) <= a < b and c > a
    with pytest.raises(abi.BsError):
        abi.bs_workspace_bytes(-1, 1, "int32")
    with pytest.raises(abi.BsError):
        abi.bs_workspace_bytes(10, 1, "none")


def test_create_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    st = abi.load().bs_create(C.byref(h), 0)
    assert st in (abi.BS_ERR_CUDA, abi.BS_ERR_INVALID_ARG)
    assert not h.value


def test_workspace_is_one_scratch_copy_plus_small_index_arrays():
    """Memory model (the paper's Exp. 2 analogue): the scratch is one copy of
    keys (and values) plus index arrays that grow with n / tile and p."""
    for kt, vt, e in (("int32", "none", 4), ("uint64", "int32", 12), ("float64", "uint64", 16)):
        for n in (2_500_000, 5_000_000, 1 << 26):
            ws = abi.bs_workspace_bytes(n, 2, kt, vt)
            assert e * n <= ws <= e * n + n // 64 + (1 << 16), (kt, vt, n, ws)
    # linear in n: equal steps of n add equal bytes (Table 2's sizes)
    steps = [abi.bs_workspace_bytes(int(2.5e6 + 5e5 * i), 2, "int32") for i in range(6)]
    diffs = np.diff(steps)
    assert diffs.max() - diffs.min() <= 1024


def _enum(src, prefix):
    return {m.group(1): int(m.group(2)) for m in re.finditer(rf"\b({prefix}\w+)\s*=\s*(-?\d+)", src)}


def test_binding_tables_match_the_header_enums():
    """The binding's option, dtype and status numbers are the header's."""
    src = open(os.path.join(ROOT, "include", "bsort.h")).read()
    opts = _enum(src, "BS_OPT_")
    assert {("BS_OPT_" + k.upper()): v for k, v in abi.OPTIONS.items()} == opts
    dts = {k: v for k, v in _enum(src, "BS_").items()
           if k in ("BS_NONE", "BS_INT32", "BS_UINT32", "BS_FLOAT32", "BS_INT64", "BS_UINT64", "BS_FLOAT64")}
    assert {("BS_" + k.upper()): v for k, v in abi.DTYPES.items()} == dts
    for name in ("BS_OK", "BS_ERR_INVALID_ARG", "BS_ERR_UNSUPPORTED_DTYPE", "BS_ERR_OUT_OF_MEMORY",
                 "BS_ERR_CUDA", "BS_ERR_TIMEOUT"):
        assert getattr(abi, name) == _enum(src, "BS_")[name], name
