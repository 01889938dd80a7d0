"""The one-exchange sort cuts sorted blocks in the library's order, not by
numeric value (CPU, gloo, world size 2 and 3): float keys with -0/+0, +-inf
and NaNs of both signs land on the right rank, so the ranks' parts,
concatenated, equal the oracle's totalOrder sort.  The order keys here come
from the oracle's codec (the GPU path uses the library's bs_order_keys)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _keys(rank, n, kind):
    from paper_1105_6040_gb300 import workloads as W
    if kind == "float32_bits":  # every bit pattern: NaNs of both signs, -0, infinities
        return W.uniform_float32_bits(n, seed=200 + rank)
    x = W.normal_float32_edges(n, seed=300 + rank)
    if kind == "float32_nans":  # a quarter NaNs of each sign (payloads from the stream)
        bits = x.view(np.uint32)
        h = W.splitmix64(400 + rank, 0, n)
        nan = (h & np.uint64(3)).astype(np.uint32)
        payload = ((h >> np.uint64(8)).astype(np.uint32) & np.uint32(0x7FFFFF)) | np.uint32(1)
        bits[nan == 0] = (np.uint32(0xFF800000) | payload)[nan == 0]   # -NaN
        bits[nan == 1] = (np.uint32(0x7F800000) | payload)[nan == 1]   # +NaN
        return x
    if kind == "float32_zeros":  # mostly -0 and +0, the pair a numeric cut would mix up
        x[: n // 2] = -0.0
        x[n // 2:: 3] = 0.0
    return x


def _cpu_sort(x):
    import oracle
    return torch.from_numpy(oracle.sort(x.numpy())[0])


def _cpu_merge(x, offsets):
    import oracle
    return torch.from_numpy(oracle.sort(x.numpy(), p=max(1, len(offsets) - 1))[0])


def _cpu_order_keys(x):
    import oracle
    codes = oracle.encode(x.numpy())  # uint64 codes of the library's order
    return torch.from_numpy((codes ^ np.uint64(1 << 63)).view(np.int64))


def _worker(rank, world, port, sizes, kind, q):
    import datetime
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1105_6040_gb300 import distributed as D
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    x = _keys(rank, sizes[rank], kind)
    part = D.exchange_sort(torch.from_numpy(x), local_sort=_cpu_sort, merge_runs=_cpu_merge,
                           order_keys=_cpu_order_keys, samples_per_rank=16)
    gathered = [None] * world
    dist.all_gather_object(gathered, part.numpy())
    if rank == 0:
        q.put(gathered)
    dist.destroy_process_group()


@pytest.mark.parametrize("world,sizes,kind", [
    (2, [5000, 7001], "float32_bits"),
    (3, [4000, 3, 6000], "float32_edges"),
    (2, [3000, 3000], "float32_zeros"),
    (2, [6000, 5000], "float32_nans"),
    (3, [2000, 4000, 3000], "float32_nans"),
])
def test_exchange_cuts_in_total_order(world, sizes, kind):
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, sizes, kind, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want, _ = oracle.sort(np.concatenate([_keys(r, sizes[r], kind) for r in range(world)]))
    got = np.concatenate(gathered)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
