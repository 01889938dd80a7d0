"""Seeded synthetic inputs for the block-decomposed sort.

This module holds only random-number generation and input layouts: no
encoding, comparison, sorting or merging.  Both the tests (CUDA path and CPU
oracle) and the benchmark draw their inputs from here, so the two sides sort
the very same bytes.

Every stream is counter based: element ``i`` of stream ``seed`` is
``splitmix64(seed + (i + 1) * 0x9E3779B97F4A7C15)`` (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), so any slice
can be regenerated on its own and the result does not depend on chunking.

The paper times "arbitrary data" (Sec. 4) and names no dataset; the shapes
below are the workloads the benchmarks use:

* int32 key sorts of 2^20 .. 2^28 keys: uniform over the full range, already
  sorted, reverse sorted, and 16 distinct values (heavy duplicates);
* stable pairs: uint64 keys (uniform, or Zipf(1.1) over 2^20 distinct keys)
  with an int32 payload equal to the original index;
* batched: segment lengths log-uniform in [lo, hi];
* serving: Poisson arrivals, float32 keys from N(0, 1) with 1% of them
  replaced by +inf, -inf, +0 or -0.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22

# per-purpose stream offsets, so one user seed yields independent streams
STREAM_KEYS = 0x0000
STREAM_ZIPF = 0x5A1F
STREAM_NORMAL_U1 = 0x1111
STREAM_NORMAL_U2 = 0x2222
STREAM_EDGES = 0x3333
STREAM_LENGTHS = 0x4444
STREAM_ARRIVALS = 0x5555
STREAM_DTYPE = 0x6666

DEFAULT_SEED = 0xB5EED000


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Elements [start, start+count) of the counter-based splitmix64 stream."""
    out = np.empty(count, dtype=np.uint64)
    s = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for c0 in range(0, count, _CHUNK):
            c1 = min(count, c0 + _CHUNK)
            i = np.arange(start + c0 + 1, start + c1 + 1, dtype=np.uint64)
            out[c0:c1] = _mix(s + i * GOLDEN)
    return out


def mix64(x: np.ndarray) -> np.ndarray:
    """The splitmix64 finaliser applied to given 64-bit words."""
    with np.errstate(over="ignore"):
        return _mix(np.asarray(x, dtype=np.uint64))


def _unit(seed: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits each."""
    return (splitmix64(seed, 0, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# --------------------------------------------------------------------------- int32 keys

def uniform_int32(n: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Uniform over the full int32 range: the low 32 bits of each draw."""
    out = np.empty(n, dtype=np.int32)
    for c0 in range(0, n, _CHUNK):
        c1 = min(n, c0 + _CHUNK)
        h = splitmix64(seed ^ STREAM_KEYS, c0, c1 - c0)
        out[c0:c1] = h.astype(np.uint32).view(np.int32)
    return out


def _s64(u: int) -> int:
    """A 64-bit pattern as the signed value torch's int64 holds."""
    u &= 0xFFFFFFFFFFFFFFFF
    return u - (1 << 64) if u >= (1 << 63) else u


def _mix_t(z):
    """splitmix64's finaliser on a torch int64 tensor (wrapping arithmetic,
    logical right shifts)."""
    def shr(x, k):
        return (x >> k) & ((1 << (64 - k)) - 1)
    z = (z ^ shr(z, 30)) * _s64(int(_M1))
    z = (z ^ shr(z, 27)) * _s64(int(_M2))
    return z ^ shr(z, 31)


def splitmix64_torch(seed: int, start: int, count: int, device="cuda"):
    """The same stream as splitmix64(), as the bits of a torch int64 tensor
    generated on `device` (for inputs too large to generate on the host)."""
    import torch
    out = torch.empty(count, dtype=torch.int64, device=device)
    s = _s64(seed)
    g = _s64(int(GOLDEN))
    chunk = 1 << 26
    for c0 in range(0, count, chunk):
        c1 = min(count, c0 + chunk)
        i = torch.arange(start + c0 + 1, start + c1 + 1, dtype=torch.int64, device=device)
        out[c0:c1] = _mix_t(i * g + s)
    return out


def uniform_int32_torch(n: int, seed: int = DEFAULT_SEED, device="cuda"):
    """uniform_int32(n, seed), generated on `device` as a torch int32 tensor."""
    import torch
    out = torch.empty(n, dtype=torch.int32, device=device)
    chunk = 1 << 26
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        h = splitmix64_torch(seed ^ STREAM_KEYS, c0, c1 - c0, device)
        out[c0:c1] = (h & 0xFFFFFFFF).to(torch.int32)  # low 32 bits, wrapped
    return out


def int32_keys_torch(dist: str, n: int, seed: int = DEFAULT_SEED, device="cuda"):
    """int32_keys(dist, n, seed), generated on `device` as a torch int32 tensor."""
    import torch
    if dist == "uniform":
        return uniform_int32_torch(n, seed, device)
    if dist in ("sorted", "reverse"):
        i = torch.arange(n, dtype=torch.int64, device=device)
        v = ((i << 32) // max(n, 1) - (1 << 31)).to(torch.int32)
        return v if dist == "sorted" else v.flip(0).contiguous()
    if dist == "dup16":
        out = torch.empty(n, dtype=torch.int32, device=device)
        chunk = 1 << 26
        for c0 in range(0, n, chunk):
            c1 = min(n, c0 + chunk)
            k = splitmix64_torch(seed ^ STREAM_KEYS, c0, c1 - c0, device) & 15
            out[c0:c1] = (k * (1 << 28) - (1 << 31)).to(torch.int32)
        return out
    raise ValueError(dist)


def uniform_uint64_torch(n: int, seed: int = DEFAULT_SEED, device="cuda"):
    """uniform_uint64(n, seed), generated on `device` (bits in a torch int64 tensor)."""
    return splitmix64_torch(seed ^ STREAM_KEYS, 0, n, device)


def sorted_int32(n: int) -> np.ndarray:
    """a_i = INT32_MIN + floor(i * 2^32 / n): strictly increasing for n <= 2^32."""
    if n == 0:
        return np.empty(0, dtype=np.int32)
    i = np.arange(n, dtype=np.uint64)
    v = (i << np.uint64(32)) // np.uint64(n)
    return (v.astype(np.int64) - 2 ** 31).astype(np.int32)


def reverse_int32(n: int) -> np.ndarray:
    return sorted_int32(n)[::-1].copy()


def dup16_int32(n: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """16 distinct values INT32_MIN + k * 2^28, k = draw & 15."""
    out = np.empty(n, dtype=np.int32)
    for c0 in range(0, n, _CHUNK):
        c1 = min(n, c0 + _CHUNK)
        k = (splitmix64(seed ^ STREAM_KEYS, c0, c1 - c0) & np.uint64(15)).astype(np.int64)
        out[c0:c1] = (k * (1 << 28) - 2 ** 31).astype(np.int32)
    return out


INT32_DISTRIBUTIONS = {
    "uniform": uniform_int32,
    "sorted": lambda n, seed=DEFAULT_SEED: sorted_int32(n),
    "reverse": lambda n, seed=DEFAULT_SEED: reverse_int32(n),
    "dup16": dup16_int32,
}


def int32_keys(dist: str, n: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    return INT32_DISTRIBUTIONS[dist](n, seed)


# --------------------------------------------------------------------------- uint64 pairs

def uniform_uint64(n: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    return splitmix64(seed ^ STREAM_KEYS, 0, n)


def zipf_uint64(n: int, seed: int = DEFAULT_SEED, s: float = 1.1,
                ranks: int = 1 << 20) -> np.ndarray:
    """Zipf(s) over `ranks` distinct keys: rank r in [1, ranks] with
    P(r) proportional to r^-s, drawn by inverting the CDF; rank r maps to the
    spread-out key mix64(r ^ 0x9E3779B97F4A7C15)."""
    w = np.arange(1, ranks + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    out = np.empty(n, dtype=np.uint64)
    for c0 in range(0, n, _CHUNK):
        c1 = min(n, c0 + _CHUNK)
        h = splitmix64(seed ^ STREAM_ZIPF, c0, c1 - c0)
        u = (h >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        r = np.minimum(np.searchsorted(cdf, u, side="right"), ranks - 1) + 1
        out[c0:c1] = mix64(r.astype(np.uint64) ^ GOLDEN)
    return out


def index_payload(n: int) -> np.ndarray:
    """int32 payload = original index (makes stability checkable exactly)."""
    return np.arange(n, dtype=np.int32)


# --------------------------------------------------------------------------- float32 keys

EDGE_VALUES = np.array([np.inf, -np.inf, 0.0, -0.0], dtype=np.float32)


def normal_float32_edges(n: int, seed: int = DEFAULT_SEED, edge_frac_pct: int = 1) -> np.ndarray:
    """N(0, 1) by Box-Muller from two counter streams; `edge_frac_pct` percent
    of the entries are replaced by +inf, -inf, +0 or -0 (chosen uniformly)."""
    out = np.empty(n, dtype=np.float32)
    for c0 in range(0, n, _CHUNK):
        c1 = min(n, c0 + _CHUNK)
        m = c1 - c0
        h1 = splitmix64(seed ^ STREAM_NORMAL_U1, c0, m)
        h2 = splitmix64(seed ^ STREAM_NORMAL_U2, c0, m)
        u1 = ((h1 >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)  # (0, 1]
        u2 = (h2 >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)
        chunk = z.astype(np.float32)
        h3 = splitmix64(seed ^ STREAM_EDGES, c0, m)
        pick = (h3 % np.uint64(100)) < np.uint64(edge_frac_pct)
        which = ((h3 >> np.uint64(32)) & np.uint64(3)).astype(np.int64)
        chunk[pick] = EDGE_VALUES[which[pick]]
        out[c0:c1] = chunk
    return out


def uniform_float32_bits(n: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Arbitrary float32 bit patterns (NaNs, subnormals, infinities included)."""
    return uniform_int32(n, seed).view(np.float32)


def uniform_float64_bits(n: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    return uniform_uint64(n, seed).view(np.float64)


# --------------------------------------------------------------------------- batches / serving

def loguniform_lengths(count: int, lo: int, hi: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """floor(exp(U(ln lo, ln hi))) clamped to [lo, hi]."""
    u = _unit(seed ^ STREAM_LENGTHS, count)
    v = np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo))))
    return np.clip(v, lo, hi).astype(np.int64)


def offsets_from_lengths(lengths: np.ndarray) -> np.ndarray:
    off = np.zeros(len(lengths) + 1, dtype=np.int64)
    np.cumsum(np.asarray(lengths, dtype=np.int64), out=off[1:])
    return off


def poisson_arrivals(rate: float, duration: float, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process of `rate` per second."""
    expect = int(rate * duration * 1.2 + 64)
    u = _unit(seed ^ STREAM_ARRIVALS, expect)
    gaps = -np.log1p(-u) / rate
    t = np.cumsum(gaps)
    while t[-1] < duration:  # extremely unlikely; extend the stream
        expect *= 2
        u = _unit(seed ^ STREAM_ARRIVALS, expect)
        t = np.cumsum(-np.log1p(-u) / rate)
    return t[t < duration]


def coin(count: int, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Fair coin flips (0/1) from their own stream (e.g. the dtype of a request)."""
    return (splitmix64(seed ^ STREAM_DTYPE, 0, count) & np.uint64(1)).astype(np.int64)
