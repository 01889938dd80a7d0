"""Build the CUDA library (libbsort.so) in-tree for sm_103a.

The translation units under csrc/ are compiled in parallel with nvcc
(-gencode arch=compute_103a,code=sm_103a) and linked into
``paper_1105_6040_gb300/_build/libbsort.so``.  A stamp of the sources' hash
skips the work when nothing changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB_NAME = "libbsort.so"
UNITS = ["bs_api.cu", "bs_u32.cu", "bs_u64.cu", "bs_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libbsort.so")


def _sources() -> list[str]:
    files = []
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            if f.endswith((".cu", ".cuh", ".h")):
                files.append(os.path.join(d, f))
    return files


def _digest() -> str:
    h = hashlib.sha256()
    for p in _sources() + [os.path.abspath(__file__)]:
        h.update(p.encode())
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def lib_path() -> str:
    return os.path.join(OUT_DIR, LIB_NAME)


def build(verbose: bool = False, force: bool = False) -> str:
    """Compile and link libbsort.so if stale; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    lib = lib_path()
    stamp = lib + ".stamp"
    key = _digest()
    if not force and os.path.exists(lib) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == key:
                return lib
    cc = nvcc()
    common = ["-std=c++17", *ARCH, "-O3", "-lineinfo", "-Xcompiler", "-fPIC",
              f"-I{INCLUDE}", f"-I{CSRC}"]

    def compile_unit(u: str) -> str:
        obj = os.path.join(OUT_DIR, u.replace(".cu", ".o"))
        cmd = [cc, *common, "-c", os.path.join(CSRC, u), "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {u}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    tmp = lib + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    with open(stamp, "w") as f:
        f.write(key)
    return lib


if __name__ == "__main__":
    import sys
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
