"""Merge phase over caller-sorted runs (bs_merge_runs) and the exchange sort
on one GPU (world size 1), against the oracle bit for bit."""
import os

import numpy as np
import pytest

import oracle
from paper_1105_6040_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sorter():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_6040_gb300.abi import Sorter
    s = Sorter(0)
    yield s
    s.close()


@pytest.mark.parametrize("lens", [
    [5000, 7001], [1, 0, 30000, 2, 0], [4096] * 7, list(range(0, 6400, 100)),
    [100000, 3, 3, 3], [0, 0, 0, 17],
], ids=["two", "skewed_empty", "seven_equal", "64_growing", "one_big", "mostly_empty"])
@pytest.mark.parametrize("dtype", ["int32", "uint64", "float32"])
def test_merge_runs_matches_oracle(sorter, lens, dtype):
    lens = np.array(lens, dtype=np.int64)
    off = W.offsets_from_lengths(lens)
    n = int(off[-1])
    x = {"int32": W.uniform_int32(n, 1) % 5000, "uint64": W.uniform_uint64(n, 2),
         "float32": W.normal_float32_edges(n, 3)}[dtype]
    runs = np.concatenate([oracle.sort(x[off[i]:off[i + 1]])[0] for i in range(lens.size)]) \
        if n else x
    if dtype == "uint64":
        d = torch.from_numpy(runs.view(np.int64)).cuda().view(torch.uint64)
    else:
        d = torch.from_numpy(runs).cuda()
    out = sorter.merge_runs(d, off.tolist())
    sorter.sync()
    got = out.view(torch.int64).cpu().numpy().view(np.uint64) if dtype == "uint64" else out.cpu().numpy()
    bits = np.uint32 if got.dtype.itemsize == 4 else np.uint64
    assert np.array_equal(got.view(bits), oracle.sort(x)[0].view(bits))


def test_merge_runs_rejects_bad_offsets(sorter):
    from paper_1105_6040_gb300 import abi
    d = torch.zeros(10, dtype=torch.int32, device="cuda")
    for bad in ([0, 5, 3, 10], [1, 10], [0, 9]):
        with pytest.raises(abi.BsError) as e:
            sorter.merge_runs(d, bad)
        assert e.value.status == abi.BS_ERR_INVALID_ARG


def test_exchange_sort_one_rank_on_gpu(sorter):
    import datetime
    import torch.distributed as dist
    from paper_1105_6040_gb300 import distributed as D
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    os.environ.setdefault("MASTER_PORT", "29561")
    dist.init_process_group("gloo", rank=0, world_size=1, timeout=datetime.timedelta(seconds=60))
    try:
        x = W.uniform_int32(300001, seed=9)
        part = D.exchange_sort(torch.from_numpy(x).cuda())
        assert np.array_equal(part.cpu().numpy(), oracle.sort(x)[0])
        val, ms, keys = D.replica_throughput(x.size, 2.0)
        assert keys == x.size and ms == 2.0
    finally:
        dist.destroy_process_group()


def test_unsorted_runs_and_overlapping_offsets_stay_in_bounds(sorter):
    """Inputs that break the sortedness a merge pass relies on (runs that are
    not sorted; overlapping segment offsets spanning many tiles) give an
    undefined output but no fault, and the handle keeps working: the
    persistent merge (forced at this size), the per-pass TMA merge and the
    plain merge kernel."""
    from paper_1105_6040_gb300 import abi
    x = W.uniform_int32(1 << 18, seed=11)
    d = torch.from_numpy(x).cuda()
    for tma, persistent in (("tma", 2), ("tma", 0), ("simple", 0)):
        abi.bs_set_option(sorter.h, "merge_kernel", tma)
        abi.bs_set_option(sorter.h, "merge_persistent", persistent)
        sorter.merge_runs(d, [0, 100003, 150000, 1 << 18])  # runs not sorted
        sorter.sync()
        bad = torch.tensor([0, 150000, 50000, 1 << 18], dtype=torch.int64, device="cuda")
        sorter.sort_segmented(d, bad)
        assert abi.bs_sync_status(sorter.h) == abi.BS_ERR_INVALID_ARG
        out = sorter.sort_keys(d, p=3)
        sorter.sync()
        assert np.array_equal(out.cpu().numpy(), np.sort(x))
    abi.bs_set_option(sorter.h, "merge_kernel", "auto")
    abi.bs_set_option(sorter.h, "merge_persistent", 1)


def _gpu_exchange_worker(rank, world, port, sizes, kind, q):
    """One rank of the exchange sort: keys on GPU 0 (shared by the ranks), the
    library's sort, order keys and merge on the device, the collectives on
    host copies (gloo)."""
    import datetime
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    from paper_1105_6040_gb300 import distributed as D
    torch.cuda.set_device(0)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=90))
    try:
        x = _exchange_keys(rank, sizes[rank], kind)
        dev = torch.from_numpy(x.view(np.int64)).cuda().view(torch.uint64) if kind == "uint64" \
            else torch.from_numpy(x).cuda()
        part = D.exchange_sort(dev)
        torch.cuda.synchronize()
        host = part.view(torch.int64).cpu().numpy().view(np.uint64) if kind == "uint64" else part.cpu().numpy()
        gathered = [None] * world
        dist.all_gather_object(gathered, host)
        if rank == 0:
            q.put(gathered)
    finally:
        dist.destroy_process_group()


def _exchange_keys(rank, n, kind):
    if kind == "int32":
        return W.uniform_int32(n, seed=600 + rank)
    if kind == "uint64":
        return W.uniform_uint64(n, seed=600 + rank)
    if kind == "float32_bits":
        return W.uniform_float32_bits(n, seed=600 + rank)   # NaNs of both signs, -0, infinities
    return W.normal_float32_edges(n, seed=600 + rank)      # +-inf, +-0 among normal values


@pytest.mark.parametrize("sizes,kind", [
    ([300001, 123457], "int32"), ([200000, 70001], "float32_bits"),
    ([150000, 150000], "float32_edges"), ([100003, 90001], "uint64"),
])
def test_exchange_sort_two_ranks_share_one_gpu(sizes, kind):
    """World size 2 through the library: two gloo processes on the one GPU,
    local sort (bs_sort_keys), splitters and cuts in the library's order
    (bs_order_keys), one all-to-all of host copies, merge of the received runs
    (bs_merge_runs); the ranks' parts concatenated equal the oracle's sort of
    both inputs, bit for bit."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_gpu_exchange_worker, args=(r, 2, port, sizes, kind, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        gathered = q.get(timeout=240)
    finally:
        for p in procs:
            p.join(timeout=120)
    for p in procs:
        assert p.exitcode == 0
    want, _ = oracle.sort(np.concatenate([_exchange_keys(r, sizes[r], kind) for r in range(2)]))
    got = np.concatenate(gathered)
    bits = np.uint32 if got.dtype.itemsize == 4 else np.uint64
    assert np.array_equal(got.view(bits), want.view(bits))
    assert all(g.size > 0 for g in gathered)  # the splitters cut the data between the ranks
