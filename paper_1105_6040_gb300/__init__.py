"""GB300-native block-decomposed sort (scatter / local sort / merge).

The compute path lives in the CUDA library built from ``csrc/`` (C-ABI declared
in ``include/bsort.h``); :mod:`.abi` is the thin ctypes binding over it.
Importing this package does not load the library: ``abi`` is imported lazily so
that :mod:`.workloads` stays usable on machines without a GPU.
"""
import importlib

__all__ = ["abi", "workloads", "batching", "serving", "autotune"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
