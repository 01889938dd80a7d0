"""Source checks of the launch discipline (CPU only).

Every kernel is launched with programmatic stream serialization
(launch_overlapped), so its CTAs may start while the kernel before it on the
stream is still running.  That is safe only if the kernel issues
griddepcontrol.wait (griddep_wait) before it touches global memory; a kernel
added without it would read its predecessor's output early.  These checks
keep both halves of that contract in the sources."""
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1105_6040_gb300", "csrc")
SOURCES = [f for f in sorted(os.listdir(CSRC)) if f.endswith((".cu", ".cuh", ".h"))]


def _read(name):
    return open(os.path.join(CSRC, name)).read()


def _match(text, i, open_ch, close_ch):
    """Index just past the bracket that closes the one at text[i]."""
    depth = 0
    while True:
        depth += {open_ch: 1, close_ch: -1}.get(text[i], 0)
        i += 1
        if depth == 0:
            return i


def _kernel_bodies(text):
    """(name, body) of every __global__ function defined in `text`."""
    out = []
    for m in re.finditer(r"__global__\s+void\s+", text):
        i = m.end()
        if text.startswith("__launch_bounds__", i):
            i = _match(text, text.index("(", i), "(", ")")
        name = re.match(r"\s*(\w+)\s*\(", text[i:])
        i = _match(text, text.index("(", i), "(", ")")  # the parameter list
        if not text[i:].lstrip().startswith("{"):
            continue  # a declaration
        j = text.index("{", i)
        out.append((name.group(1), text[j:_match(text, j, "{", "}")]))
    return out


def test_every_kernel_waits_for_its_predecessor_first():
    kernels = [kb for name in SOURCES for kb in _kernel_bodies(_read(name))]
    assert len(kernels) >= 16 and any(n == "merge_tma_kernel" for n, _ in kernels)
    for name, body in kernels:
        assert "griddep_wait();" in body, name
        # nothing global is read or written before the wait: only shared
        # memory set-up (and barrier initialisation) may precede it
        head = body[: body.index("griddep_wait();")]
        for bad in ("atomicAdd", "g.tseg", "g.off", "in_k[", "split[", "*ntiles_total", "off[", "out["):
            assert bad not in head, (name, bad)


def test_every_launch_goes_through_launch_overlapped():
    for name in SOURCES:
        text = re.sub(r"//[^\n]*", "", _read(name))
        assert "<<<" not in text, name
