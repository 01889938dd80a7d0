"""Multi-rank paths on the CPU with the gloo backend (world sizes 2 and 3):
replica timing aggregation, the one-exchange distributed sort (checked
against the oracle on the concatenated input), and a failed rank surfacing
as an error on the others instead of a hang."""
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


def _init(rank, world, port, timeout_s=60):
    import datetime
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=timeout_s))


def _cpu_sort(x):
    import oracle
    return torch.from_numpy(oracle.sort(x.numpy())[0])


def _cpu_merge(x, offsets):
    import oracle
    # merging sorted runs yields the sorted whole; the oracle sorts the
    # concatenation with one block per run
    a = x.numpy()
    return torch.from_numpy(oracle.sort(a, p=max(1, len(offsets) - 1))[0])


def _worker_exchange(rank, world, port, sizes, dtype, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1105_6040_gb300 import distributed as D
    from paper_1105_6040_gb300 import workloads as W
    _init(rank, world, port)
    n = sizes[rank]
    x = W.uniform_int32(n, seed=100 + rank) if dtype == "int32" else \
        W.uniform_uint64(n, seed=100 + rank).view(np.int64)
    if dtype == "dup":
        x = (W.uniform_int32(n, seed=100 + rank) % 7).astype(np.int32)
    part = D.exchange_sort(torch.from_numpy(x), local_sort=_cpu_sort, merge_runs=_cpu_merge,
                           samples_per_rank=16)
    gathered = [None] * world
    dist.all_gather_object(gathered, part.numpy())
    val, ms, keys = D.replica_throughput(n, 10.0 + rank)
    if rank == 0:
        q.put((gathered, val, ms, keys))
    dist.destroy_process_group()


@pytest.mark.parametrize("world,sizes,dtype", [
    (2, [5000, 7001], "int32"),
    (3, [4096, 1, 9999], "int64"),
    (3, [3000, 0, 2500], "dup"),
])
def test_exchange_sort_matches_oracle(world, sizes, dtype):
    import oracle
    from paper_1105_6040_gb300 import workloads as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_worker_exchange, args=(r, world, port, sizes, dtype, q))
             for r in range(world)]
    for p in procs:
        p.start()
    gathered, val, ms, keys = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    parts = []
    for r in range(world):
        n = sizes[r]
        x = W.uniform_int32(n, seed=100 + r) if dtype == "int32" else \
            W.uniform_uint64(n, seed=100 + r).view(np.int64)
        if dtype == "dup":
            x = (W.uniform_int32(n, seed=100 + r) % 7).astype(np.int32)
        parts.append(x)
    want, _ = oracle.sort(np.concatenate(parts))
    got = np.concatenate(gathered)
    assert np.array_equal(got, want)
    # rank order is key order, and no rank overlaps the next
    for a, b in zip(gathered, gathered[1:]):
        if a.size and b.size:
            assert a[-1] <= b[0]
    # replica aggregation: total keys over the slowest rank's time
    assert keys == sum(sizes) and ms == 10.0 + (world - 1)
    assert abs(val - sum(sizes) / (ms * 1e-3) / 1e9) < 1e-12


def _worker_fail(rank, world, port, q):
    import time
    _init(rank, world, port, timeout_s=10)
    if rank == 1:
        raise SystemExit(3)  # this rank dies before the collective
    t0 = time.time()
    try:
        dist.all_reduce(torch.ones(1))
        q.put(("no error", time.time() - t0))
    except Exception as e:  # the survivor learns of it on the host
        q.put((type(e).__name__, time.time() - t0))


def test_a_failed_rank_surfaces_as_an_error_not_a_hang():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_worker_fail, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    kind, secs = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert kind != "no error"
    assert secs < 60
