"""Several GPUs: replicas, and the one-exchange sort of one array spread over ranks.

The paper's paradigm partitions the data (Sec. 3.2, Fig. 1): each process
sorts its block, then the blocks are merged.  Across GPUs that becomes:

* replicas (what the benchmark runs): every rank sorts its own independent
  array; nothing crosses ranks on the data path.  ``replica_throughput``
  combines the ranks' timings (max over ranks) into one whole-job figure.
* one distributed array (``exchange_sort``): rank r holds block r.
  1. local sort of the block (the sort phase);
  2. splitters: every rank contributes evenly spaced samples of its sorted
     block, all ranks gather them and take G-1 evenly spaced splitters of
     the sorted samples;
  3. one exchange: rank r sends to rank q the keys k with
     splitter[q-1] <= k < splitter[q] (all_to_all_single, variable sizes);
  4. rank q merges the G sorted runs it received (the merge phase,
     ``bs_merge_runs`` on the GPU).
  Afterwards the ranks' outputs, concatenated in rank order, are the sorted
  whole.  This replaces the log2 G rounds of pairwise merges that Fig. 1
  would take across processes by a single all-to-all.

Keys: every dtype the library sorts.  Splitters are chosen, and sorted
blocks cut at them, in the library's own order: on the GPU through its order
keys (bs_order_keys: each key's order-preserving code as a signed 64-bit
integer, so floating point is cut by IEEE 754 totalOrder, -0 before +0, NaNs
by payload); host tensors of signed integer dtypes use their numeric order,
other host dtypes need an ``order_keys`` function.  Collectives run on the
process group's backend: with NCCL on the device tensors, with gloo through
host copies (keys stay on the device for the sorts), so ranks that share one
GPU can run the whole path, as the tests do.
"""
from __future__ import annotations

import numpy as np


def replica_throughput(keys_local: int, ms_local: float, group=None, device=None):
    """Whole-job throughput of independent replicas: (Gkeys/s, max ms, total keys)."""
    import torch
    import torch.distributed as dist
    dev = device if device is not None else "cpu"
    t = torch.tensor([ms_local], dtype=torch.float64, device=dev)
    k = torch.tensor([keys_local], dtype=torch.int64, device=dev)
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
        dist.all_reduce(k, op=dist.ReduceOp.SUM, group=group)
    ms, keys = float(t.item()), int(k.item())
    return keys / (ms * 1e-3) / 1e9, ms, keys


def _gpu_local_sort(x):
    from .abi import Sorter
    s = _sorter(x.device)
    out = s.sort_keys(x.contiguous(), p=1)
    return out


def _gpu_merge_runs(x, offsets):
    s = _sorter(x.device)
    return s.merge_runs(x.contiguous(), [int(o) for o in offsets])


def _order_keys(x):
    """int64 keys whose (signed) order is the library's sort order of x."""
    import torch
    if x.is_cuda:
        from .abi import order_keys
        return order_keys(x.contiguous())
    if x.dtype in (torch.int8, torch.int16, torch.int32, torch.int64):
        return x.to(torch.int64)  # numeric order is the sort order
    raise ValueError(f"host tensors of dtype {x.dtype} need an order_keys function")


def _comm(t, group):
    """The tensor a collective of this group can take: gloo works on host
    tensors only, so device tensors go through host memory."""
    import torch.distributed as dist
    if t.is_cuda and dist.get_backend(group) == "gloo":
        return t.cpu()
    return t


_SORTERS = {}


def _sorter(device):
    from .abi import Sorter
    key = str(device)
    if key not in _SORTERS:
        _SORTERS[key] = Sorter(device)
    return _SORTERS[key]


def choose_splitters(sorted_local, group=None, samples_per_rank: int = 64, local_sort=None):
    """G-1 splitters from evenly spaced samples of every rank's sorted block
    (keys of any ordered dtype: here, order keys)."""
    import torch
    import torch.distributed as dist
    G = dist.get_world_size(group)
    n = sorted_local.numel()
    s = samples_per_rank
    dev = sorted_local.device
    if n > 0:
        pos = torch.div((torch.arange(1, s + 1, device=dev) * n), s + 1,
                        rounding_mode="floor").clamp(max=n - 1)
        samp = sorted_local[pos]
        cnt = torch.tensor([s], device=dev)
    else:
        samp = torch.zeros(s, dtype=sorted_local.dtype, device=dev)
        cnt = torch.tensor([0], device=dev)
    samp, cnt = _comm(samp, group), _comm(cnt, group)
    all_samp = [torch.empty_like(samp) for _ in range(G)]
    all_cnt = [torch.empty_like(cnt) for _ in range(G)]
    dist.all_gather(all_samp, samp, group=group)
    dist.all_gather(all_cnt, cnt, group=group)
    pool = torch.cat([a[:int(c.item())] for a, c in zip(all_samp, all_cnt)]).to(dev)
    pool = (local_sort or _gpu_local_sort)(pool.contiguous())  # G * samples_per_rank keys
    if pool.numel() == 0:
        return pool
    idx = torch.tensor([(j * pool.numel()) // G for j in range(1, G)], device=pool.device)
    return pool[idx]


def exchange_sort(local, group=None, local_sort=None, merge_runs=None, order_keys=None,
                  samples_per_rank: int = 64):
    """Sort a block-distributed array with one all-to-all exchange.

    local: this rank's keys (1-D tensor: on the GPU, or on the host with a
    gloo group).  local_sort(x) -> sorted x; merge_runs(x, offsets) -> sorted
    x from sorted runs; order_keys(x) -> int64 keys in x's sort order
    (defaults: the library's bs_sort_keys, bs_merge_runs and bs_order_keys on
    the GPU).  Returns this rank's part of the sorted whole (rank order = key
    order)."""
    import torch
    import torch.distributed as dist
    local_sort = local_sort or _gpu_local_sort
    merge_runs = merge_runs or _gpu_merge_runs
    order_keys = order_keys or _order_keys
    G = dist.get_world_size(group)
    srt = local_sort(local)
    if G == 1:
        return srt
    ordk = order_keys(srt)  # nondecreasing int64, the library's order
    spl = choose_splitters(ordk, group, samples_per_rank, local_sort)
    if spl.numel() != G - 1:
        return srt  # no rank holds any key
    # bucket q gets splitter[q-1] <= key < splitter[q] (in the library's order)
    cuts = torch.searchsorted(ordk, spl, right=False)
    edges = torch.cat([torch.zeros(1, dtype=torch.int64, device=srt.device), cuts.to(torch.int64),
                       torch.tensor([srt.numel()], dtype=torch.int64, device=srt.device)])
    send = _comm((edges[1:] - edges[:-1]).to(torch.int64), group)
    recv = torch.empty_like(send)
    dist.all_to_all_single(recv, send, group=group)
    send_l, recv_l = send.tolist(), recv.tolist()
    # the keys travel as bits of the same-size signed type (gloo has no
    # unsigned 64-bit collectives); only their bits matter here
    wire = {torch.uint64: torch.int64, torch.uint32: torch.int32}.get(srt.dtype, srt.dtype)
    payload = _comm(srt.view(wire), group)
    out = torch.empty(int(sum(recv_l)), dtype=wire, device=payload.device)
    dist.all_to_all_single(out, payload, output_split_sizes=recv_l, input_split_sizes=send_l, group=group)
    out = out.to(srt.device).view(srt.dtype)
    offsets = np.concatenate([[0], np.cumsum(recv_l)]).astype(np.int64)
    if out.numel() == 0:
        return out
    return merge_runs(out, offsets)
