"""Compile the CPU oracle (plain C) into a shared library with gcc.

Test infrastructure: the oracle is loaded only by the tests, the smoke check and
the benchmark's CPU-baseline leg.  ``build(mutation=k)`` builds a variant with
planted mistake ``k`` (see ORC_MUT in bs_oracle.c) for the pin-strength tests.
"""
from __future__ import annotations

import hashlib
import os
import subprocess
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "bs_oracle.c")
HDR = os.path.join(HERE, "bs_oracle.h")
OUT_DIR = os.path.join(HERE, "_build")


def _digest() -> str:
    h = hashlib.sha256()
    for p in (SRC, HDR, __file__):
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def build(mutation: int = 0, out_dir: str | None = None) -> str:
    """Build (if stale) and return the path of the oracle shared library."""
    out_dir = out_dir or OUT_DIR
    os.makedirs(out_dir, exist_ok=True)
    name = "libbs_oracle.so" if mutation == 0 else f"libbs_oracle_mut{mutation}.so"
    lib = os.path.join(out_dir, name)
    stamp = lib + ".stamp"
    key = f"{_digest()}:{mutation}"
    if os.path.exists(lib) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == key:
                return lib
    fd, tmp = tempfile.mkstemp(suffix=".so", dir=out_dir)
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-Wall",
           f"-DORC_MUT={int(mutation)}", SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    with open(stamp, "w") as f:
        f.write(key)
    return lib


if __name__ == "__main__":
    print(build())
