#!/usr/bin/env python3
"""Benchmark: block-decomposed int32 key sort on GB300 (Gkeys/s, % of HBM roofline).

Workload (default): 2^28 uniform int32 keys from the seeded counter-based
generator, split into p = 2 blocks (the paper's dual-core decomposition), sorted
out of place through the C ABI (bs_sort_keys) on torch's current stream.
One step = one whole sort: scatter bounds, tile-sort pass, in-block merge
passes, cross-block merge round.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (under torchrun) runs N independent replicas (each rank sorts its own
array; weak scaling, no collective on the data path); timing is the max over
ranks.  --impl reference times the CPU oracle (the paper's scatter / merge-sort
/ merge-tree paradigm in plain C) on the host cores over a bounded sample.

Prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gkeys/s and % HBM roofline, 2^28 int32 on 1 GB300"
UNIT = "Gkeys/s"
FALLBACK_HBM_GBS = 6800.0
SEED = 0xB5EED000


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["keys", "pairs", "batched", "serving", "memory", "psweep",
                                           "localsort"],
                    default="keys",
                    help="keys: one 2^log2n int32 array (the headline); pairs: 2^pairs-log2n "
                         "uint64 keys with int32 index payloads (stable); batched: many "
                         "arrays of log-uniform length in one graph-captured segmented sort")
    ap.add_argument("--pairs-log2n", type=int, default=27)
    ap.add_argument("--pairs-dist", default="uniform", choices=["uniform", "zipf"])
    ap.add_argument("--pairs-tile-log2", type=int, default=13)
    ap.add_argument("--segments", type=int, default=20000)
    ap.add_argument("--seg-lo", type=int, default=16)
    ap.add_argument("--seg-hi-log2", type=int, default=17)
    ap.add_argument("--per-array-rounds", type=int, default=2)
    ap.add_argument("--merge-vt", type=int, default=0, choices=[0, 8, 16, 32])
    ap.add_argument("--merge-tile-log2", type=int, default=0, choices=[0, 11, 12, 13],
                    help="merge-pass tile 2^k keys (0: the sort tile)")
    ap.add_argument("--merge-consumer", type=int, default=0, choices=[0, 1])
    ap.add_argument("--duration", type=float, default=60.0, help="serving: seconds of arrivals")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: requests per second")
    ap.add_argument("--streams", type=int, default=4, help="serving: execution slots")
    ap.add_argument("--log2n", type=int, default=28)
    ap.add_argument("--p", type=int, default=2)
    ap.add_argument("--dist", default="uniform", choices=["uniform", "sorted", "reverse", "dup16"])
    ap.add_argument("--dists", default="",
                    help="psweep: comma-separated distributions (default: --dist)")
    ap.add_argument("--tile-log2", type=int, default=13,
                    help="sort-phase tile 2^k keys (the bench default: 8192-key sort and merge tiles)")
    ap.add_argument("--merge", choices=["auto", "simple", "tma"], default="auto",
                    help="merge-pass kernel (auto: TMA pipeline where it fits)")
    ap.add_argument("--e2e-steps", type=int, default=-1,
                    help="steps of the end-to-end record (-1: --steps; 0: none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra records of the default run (batched, pairs, serving)")
    ap.add_argument("--serving-extra-s", type=float, default=10.0,
                    help="seconds of arrivals in the default run's serving record")
    ap.add_argument("--cpu-sample-log2", type=int, default=26)
    return ap.parse_args()


# ---------------------------------------------------------------- environment helpers

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_digest() -> str:
    """Hash of the device code (the kernels live in csrc/bs_device.cuh and
    csrc/bs_persist.cuh): a recorded ncu traffic figure is used only while
    this hash is unchanged."""
    h = hashlib.sha256()
    for name in ("bs_device.cuh", "bs_persist.cuh"):
        with open(os.path.join(ROOT, "paper_1105_6040_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_from_profiles(kernel: str, workload: str):
    """Per-launch DRAM bytes of `kernel` recorded under profiles/ by an ncu
    capture of the current sources, or None when absent or stale."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    digest = kernel_digest()
    pat = re.compile(r"traffic:\s*kernel=(\S+)\s+workload=(\S+)\s+bytes_per_launch=(\d+)"
                     r"(?:\s+passes=\d+)?\s+sources=(\w+)")
    for name in sorted(os.listdir(pdir)):
        if not name.endswith((".md", ".txt")):
            continue
        with open(os.path.join(pdir, name)) as f:
            for m in pat.finditer(f.read()):
                if m.group(1) == kernel and m.group(2) == workload and m.group(4) == digest:
                    return int(m.group(3))
    return None


def instructions_from_profiles(kernel: str):
    """Thread-instructions per key of `kernel` recorded under profiles/ by an
    ncu capture of the current sources, or None when absent or stale."""
    pdir = os.path.join(ROOT, "profiles")
    if not os.path.isdir(pdir):
        return None
    digest = kernel_digest()
    pat = re.compile(r"instructions:\s*kernel=(\S+)\s+thread_instructions_per_key=([0-9.]+)\s+sources=(\w+)")
    for name in sorted(os.listdir(pdir)):
        if not name.endswith((".md", ".txt")):
            continue
        with open(os.path.join(pdir, name)) as f:
            for m in pat.finditer(f.read()):
                if m.group(1) == kernel and m.group(3) == digest:
                    return float(m.group(2))
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        sm = [float(r[1]) for r in rows if _num(r[1])]
        mx = [float(r[2]) for r in rows if _num(r[2])]
        power = [float(r[3]) for r in rows if _num(r[3])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        # "under load": the samples at the busy end of the distribution
        load = [s for s in sm if s >= 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(power) if power else None,
                "samples": len(rows), "reasons": reasons}


def _num(s):
    try:
        float(s)
        return True
    except ValueError:
        return False


# ---------------------------------------------------------------- inputs

def make_keys(args, rank: int):
    from paper_1105_6040_gb300 import workloads as W
    return W.int32_keys(args.dist, 1 << args.log2n, seed=SEED + rank)


def workload_name(args) -> str:
    return f"int32 key sort, 2^{args.log2n} {args.dist} keys, p={args.p} blocks"


def config(args):
    return {"workload": workload_name(args), "n": 1 << args.log2n, "p": args.p,
            "dist": args.dist, "key_dtype": "int32", "tile_keys": 1 << args.tile_log2,
            "merge_kernel": args.merge, "merge_vt": args.merge_vt or 32,
            "merge_tile_keys": 1 << (args.merge_tile_log2 or args.tile_log2),
            "merge_consumer": ["thread sequential merge", "warp bitonic"][args.merge_consumer],
            "seed": SEED, "l2": "inputs (4 B x n = 1 GiB at 2^28) larger than the 129 MB L2; no flush",
            "stream": "torch current stream", "out_of_place": True,
            "check": "warm-up output checked by the library's device checkers (bs_check_keys): "
                     "nondecreasing, both multiset hashes equal to the input's"}


# ---------------------------------------------------------------- CPU oracle (baseline / reference arm)

def oracle_rate(keys, repeats_s: float = 10.0, min_runs: int = 1):
    """Time the CPU oracle on `keys` with one block and one thread per host core."""
    import oracle
    cores = os.cpu_count() or 1
    oracle.load()
    runs, t_total = 0, 0.0
    while runs < min_runs or t_total < repeats_s:
        t0 = time.perf_counter()
        oracle.sort(keys, p=cores, threads=cores)
        t_total += time.perf_counter() - t0
        runs += 1
    return keys.size * runs / t_total / 1e9, cores, runs, t_total


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1105_6040_gb300 import workloads as W
    sample_log2 = min(args.log2n, 22)
    keys = _first_keys(args, 1 << sample_log2)
    cores = os.cpu_count() or 1
    oracle.load()
    for _ in range(args.warmup):
        oracle.sort(keys, p=cores, threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.sort(keys, p=cores, threads=cores)
    dt = time.perf_counter() - t0
    value = keys.size * args.steps / dt / 1e9
    sample = (f"first 2^{sample_log2} keys of the 2^{args.log2n}-key workload per step; "
              f"oracle p={cores} blocks, {cores} threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic", "config": config(args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _first_keys(args, count):
    from paper_1105_6040_gb300 import workloads as W
    if args.dist in ("uniform", "dup16"):
        return W.int32_keys(args.dist, count, seed=SEED)  # counter-based: a prefix of the stream
    full = W.int32_keys(args.dist, 1 << args.log2n, seed=SEED)
    return full[:count].copy()


def gpu_local_cpus(device):
    """The host CPUs next to the GPU (its PCI device's local_cpulist in sysfs)
    and its NUMA node, or (None, None): page-locked buffers allocated from
    those CPUs land in the memory nearest the GPU."""
    try:
        import torch
        pr = torch.cuda.get_device_properties(device)
        dev = f"/sys/bus/pci/devices/{pr.pci_domain_id:04x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
        txt = open(dev + "/local_cpulist").read().strip()
        cpus = set()
        for part in txt.split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        node = open(dev + "/numa_node").read().strip()
        return (cpus or None), node
    except Exception:
        return None, None


def pass_counts(kernels, bytes_per_pass):
    """Passes per sort (each reads and writes every item once), merge passes
    per merge launch, and the merge kernel's name: one persistent launch runs
    every merge level, the per-pass path one launch per level."""
    ts = kernels.get("tile_sort", {})
    mg = kernels.get("merge", {})
    per_step = (ts.get("bytes_per_launch", 0) * ts.get("launches_per_step", 0)
                + mg.get("bytes_per_launch", 0) * mg.get("launches_per_step", 0))
    merge_per_launch = mg.get("bytes_per_launch", 0) / bytes_per_pass
    name = "merge_persist_kernel" if merge_per_launch > 1.5 else "merge_tma_kernel"
    return per_step / bytes_per_pass, merge_per_launch, name


def extra_records(args):
    """The records of the default run besides the headline: batched segmented
    sorts (lengths log-uniform in [16, 2^17] -- about 2^28 keys -- and in
    [16, 2^20] as the workload states it, about 1.9e9 keys) against one call per
    array, 2^27 stable uint64+int32 pairs, and a short serving run.  Inputs
    are made on the GPU by the seeded generators (the same bits as the host
    ones)."""
    import argparse as _ap
    import torch
    out = {}

    def sub(**kw):
        a = _ap.Namespace(**vars(args))
        a.device_gen = True
        for k, v in kw.items():
            setattr(a, k, v)
        return a

    def keep(rec, keys):
        return {k: rec[k] for k in keys if k in rec}

    common = ("metric", "value", "unit", "ms_per_step", "steps", "warmup", "config", "clocks")
    for name, hi in (("batched_2e17", 17), ("batched_2e20", 20)):
        rec = run_batched(sub(seg_hi_log2=hi, steps=5 if hi == 17 else 3, warmup=2,
                              per_array_rounds=1))
        out[name] = keep(rec, common + ("per_array", "speedup_vs_per_array", "kernels_one_run"))
        torch.cuda.empty_cache()
    rec = run_pairs(sub(pairs_log2n=27, pairs_dist="uniform", steps=5, warmup=2, p=2))
    out["pairs"] = keep(rec, common + ("roofline", "kernels", "checked"))
    torch.cuda.empty_cache()
    rec = run_serving(sub(duration=args.serving_extra_s))
    out["serving"] = keep(rec, common + ("p50_ms", "p99_ms", "serving", "offered_gkeys_per_s"))
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- our arm

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1105_6040_gb300 import abi

    rank, world, local = dist_env()
    if world != args.gpus:
        raise SystemExit(f"--gpus {args.gpus} but WORLD_SIZE={world}")
    if not torch.cuda.is_available():
        raise SystemExit("no CUDA device: the benchmark measures the GPU path only")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    n = 1 << args.log2n
    keys_h = make_keys(args, rank)
    # the CPU baseline copy (a prefix of the same workload) is taken before any big GPU work
    cpu_sample = keys_h[: 1 << min(args.cpu_sample_log2, args.log2n)].copy()

    sorter = abi.Sorter(local, tile_log2=args.tile_log2, merge_kernel=args.merge,
                        merge_vt=args.merge_vt, merge_tile_log2=args.merge_tile_log2,
                        merge_consumer=args.merge_consumer)
    d_in = torch.from_numpy(keys_h).cuda()
    d_out = torch.empty_like(d_in)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    def step():
        abi.bs_sort_keys(sorter.h, d_in.data_ptr(), d_out.data_ptr(), n, "int32", args.p, sp)

    for _ in range(args.warmup):
        step()
    sorter.sync()
    # correctness of the warm-up output: the library's device checkers (one
    # pass each, outside the timed regions) -- sorted, same multiset of codes
    chk_in, chk_out = abi.check_keys(d_in), abi.check_keys(d_out)
    assert chk_out["first_unsorted"] == -1, "output not sorted"
    assert (chk_out["hash_a"], chk_out["hash_b"]) == (chk_in["hash_a"], chk_in["hash_b"]), \
        "output not a permutation of the input"

    # ---- timed region A: K whole sorts, CUDA events on the launching stream
    abi.bs_launch_stats(sorter.h, reset=True, with_bytes=False)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    barrier()
    ms_total = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    counts, _ = abi.bs_launch_stats(sorter.h, reset=True, with_bytes=False)
    launches = int(sum(counts.values()))
    t = torch.tensor([ms_total], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    ms_step = ms_max / args.steps
    value = world * n * args.steps / (ms_max * 1e-3) / 1e9

    # ---- timed region B: same steps with a CUDA event pair around every launch
    kb = min(args.steps, 20)
    abi.bs_launch_stats(sorter.h, reset=True)
    abi.bs_set_option(sorter.h, "count_bytes", 1)
    sorter.set_timing(True)
    barrier()
    for _ in range(kb):
        step()
    barrier()
    sorter.set_timing(False)
    abi.bs_set_option(sorter.h, "count_bytes", 0)
    kms, kn = sorter.kernel_times()
    kcounts, kbytes = abi.bs_launch_stats(sorter.h, reset=True)
    peak, peak_src = load_peak()
    kernels = {}
    for cls in ("tile_sort", "merge", "partition", "setup"):
        if kn[cls]:
            avg_ms = kms[cls] / kn[cls]
            per_launch = kbytes[cls] / kn[cls]
            kernels[cls] = {"launches_per_step": kn[cls] / kb, "ms_per_launch": avg_ms,
                            "bytes_per_launch": per_launch,
                            "gbs": per_launch / (avg_ms * 1e-3) / 1e9 if per_launch else None}
    # the tile sort is bound by instruction issue, not HBM: its issue roofline
    # (4 schedulers x 32 lanes per SM per clock, at the sampled SM clock)
    ipk = instructions_from_profiles("tile_sort_kernel")
    if "tile_sort" in kernels and ipk and clk.get("sm_mhz"):
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        issue_peak = sms * 4 * 32 * clk["sm_mhz"] * 1e6
        ach = ipk * n / (kernels["tile_sort"]["ms_per_launch"] * 1e-3)
        kernels["tile_sort"]["roofline"] = {
            "bound": "alu", "unit": "thread-instructions/s", "achieved": ach, "peak": issue_peak,
            "frac": ach / issue_peak, "thread_instructions_per_key": ipk,
            "peak_source": f"issue peak: {sms} SMs x 4 schedulers x 32 lanes x {clk['sm_mhz']:g} MHz"}
    dom = max(("tile_sort", "merge"), key=lambda c: kms[c])
    achieved = kernels[dom]["gbs"]
    passes, merge_passes, merge_name = pass_counts(kernels, 2 * 4 * n)
    traffic = traffic_from_profiles(merge_name if dom == "merge" else "tile_sort_kernel",
                                    f"int32_2e{args.log2n}_p{args.p}_{args.dist}")
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": (f"merge phase ({merge_name}: {merge_passes:g} passes per launch)"
                           if dom == "merge" else "tile sort"),
                "peak_source": f"{peak_src} (copy bandwidth)",
                "passes_per_step": passes,
                "end_to_end_frac": passes * 2 * 4 * n / (ms_step * 1e-3) / 1e9 / peak}

    # ---- end to end through the host-memory entry points (pinned host memory):
    # every step copies its input in from host memory and its sorted output
    # back; bs_sort_keys_host_async pipelines successive steps on the handle
    # (step k+1's copy in and step k-1's copy out overlap step k's sort)
    e2e = None
    e2e_steps = args.steps if args.e2e_steps < 0 else args.e2e_steps
    sync_steps = min(e2e_steps, 20)
    if e2e_steps > 0:
        # host buffers from the CPUs next to the GPU (its NUMA node's memory)
        near, node = gpu_local_cpus(local)
        old_aff = os.sched_getaffinity(0)
        if near and (near & old_aff):
            os.sched_setaffinity(0, near & old_aff)
        h_in = torch.from_numpy(keys_h).pin_memory()
        h_outs = [torch.empty_like(h_in).pin_memory() for _ in range(2)]

        def e2e_round(k):
            sorter.sort_keys_host_async(h_in, h_outs[k % 2], p=args.p, stream=stream)

        for k in range(4):
            e2e_round(k)
        sorter.sync()
        barrier()
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            e2e_round(k)
        sorter.sync()
        dt = torch.tensor([time.perf_counter() - t0], dtype=torch.float64, device="cuda")
        if world > 1:
            dist.all_reduce(dt, op=dist.ReduceOp.MAX)
        for o in h_outs[: min(2, e2e_steps)]:
            o = o.numpy()
            assert np.all(o[1:] >= o[:-1])
        # one synchronous call after another, for comparison (no overlap)
        for _ in range(2):
            abi.bs_sort_keys_host(sorter.h, h_in.data_ptr(), h_outs[0].data_ptr(), n, "int32", args.p)
        t1 = time.perf_counter()
        for _ in range(sync_steps):
            abi.bs_sort_keys_host(sorter.h, h_in.data_ptr(), h_outs[0].data_ptr(), n, "int32", args.p)
        dt_sync = time.perf_counter() - t1
        o = h_outs[0].numpy()
        assert np.all(o[1:] >= o[:-1])
        os.sched_setaffinity(0, old_aff)
        e2e = {"value": world * n * e2e_steps / float(dt.item()) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 4 * n,
               "host_buffers": {"gpu_numa_node": node,
                                "cpus": (f"{min(near)}-{max(near)} ({len(near)})" if near else None)},
               "api": "bs_sort_keys_host_async, one call per step on one handle, then "
                      "bs_sync_status (page-locked host buffers; each step's input copied in and "
                      "its sorted output copied out on the copy engines, overlapping the sorts "
                      "of the steps before and after it)",
               "steps": e2e_steps,
               "sync_calls": {"value": world * n * sync_steps / dt_sync / 1e9, "unit": UNIT,
                              "steps": sync_steps,
                              "api": "bs_sort_keys_host, one call after another (the sort phase "
                                     "reads the input and the last merge pass writes the output "
                                     "across the host link)"}}
        del h_in, h_outs

    sorter.close()
    del d_in, d_out
    torch.cuda.empty_cache()

    # ---- the metric's other clauses, each measured in this same run with its own
    # clock samples (N = 1 only): batched vs per-array at both segment-length
    # ranges, the stable pairs workload, and a short serving run (p50/p99)
    extras = None
    if world == 1 and not args.no_extras:
        extras = extra_records(args)

    # ---- CPU baseline: the oracle on this host's cores, rank 0 at N=1 only
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, cores, runs, secs = oracle_rate(cpu_sample)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first 2^{min(args.cpu_sample_log2, args.log2n)} keys of the workload, "
                         f"{runs} run(s) in {secs:.1f} s; oracle p={cores} blocks, {cores} threads"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": config(args), "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "launches_per_step": launches / args.steps,
            "clocks": clk, "kernels": kernels,
        }
        if extras is not None:
            line["extras"] = extras
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- stable pairs workload

def run_pairs(args):
    """2^27 uint64 keys (uniform, or Zipf(1.1) over 2^20 distinct keys) with an
    int32 payload = original index, p = 2, sorted stably through bs_sort_pairs.
    12 bytes move per item per pass."""
    import numpy as np
    import torch

    from paper_1105_6040_gb300 import abi
    from paper_1105_6040_gb300 import workloads as W

    n = 1 << args.pairs_log2n
    sorter = abi.Sorter(0, tile_log2=args.pairs_tile_log2, merge_kernel=args.merge, merge_vt=args.merge_vt,
                        merge_consumer=args.merge_consumer)  # merge tile: the library's choice
    if getattr(args, "device_gen", False) and args.pairs_dist == "uniform":
        dk = W.uniform_uint64_torch(n, seed=SEED).view(torch.uint64)  # the same bits, made on the GPU
        dv = torch.arange(n, dtype=torch.int32, device="cuda")
    else:
        keys_h = (W.uniform_uint64(n, seed=SEED) if args.pairs_dist == "uniform"
                  else W.zipf_uint64(n, seed=SEED))
        vals_h = W.index_payload(n)
        dk, dv = torch.from_numpy(keys_h).cuda(), torch.from_numpy(vals_h).cuda()
    ko, vo = torch.empty_like(dk), torch.empty_like(dv)
    stream = torch.cuda.current_stream()

    def step():
        abi.bs_sort_pairs(sorter.h, dk.data_ptr(), ko.data_ptr(), dv.data_ptr(), vo.data_ptr(), n,
                          "uint64", "int32", args.p, stream.cuda_stream)

    for _ in range(args.warmup):
        step()
    sorter.sync()
    # the output is the stable sort iff: the payload is a permutation, every key
    # travelled with its payload, keys are nondecreasing, equal keys keep order
    idx = vo.long()
    assert bool((torch.bincount(idx, minlength=n) == 1).all()), "payload not a permutation"
    assert torch.equal(ko.view(torch.int64), dk.view(torch.int64)[idx]), "key and payload parted"
    code = ko.view(torch.int64) ^ torch.tensor(-(1 << 63), dtype=torch.int64, device="cuda")
    assert bool((code[1:] >= code[:-1]).all()), "keys not sorted"
    eq = code[1:] == code[:-1]
    assert bool((vo[1:][eq] > vo[:-1][eq]).all()), "not stable"
    del idx, code, eq

    abi.bs_launch_stats(sorter.h, reset=True, with_bytes=False)
    clocks = ClockSampler(0)
    clocks.start()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    clk = clocks.stop()
    counts, _ = abi.bs_launch_stats(sorter.h, reset=True, with_bytes=False)
    kb = min(args.steps, 10)
    abi.bs_launch_stats(sorter.h, reset=True)
    abi.bs_set_option(sorter.h, "count_bytes", 1)
    sorter.set_timing(True)
    for _ in range(kb):
        step()
    torch.cuda.synchronize()
    sorter.set_timing(False)
    abi.bs_set_option(sorter.h, "count_bytes", 0)
    kms, kn = sorter.kernel_times()
    _, kbytes = abi.bs_launch_stats(sorter.h, reset=True)
    peak, peak_src = load_peak()
    kernels = {}
    for cls in ("tile_sort", "merge", "partition", "setup"):
        if kn[cls]:
            avg = kms[cls] / kn[cls]
            per = kbytes[cls] / kn[cls]
            kernels[cls] = {"launches_per_step": kn[cls] / kb, "ms_per_launch": avg, "bytes_per_launch": per,
                            "gbs": per / (avg * 1e-3) / 1e9 if per else None}
    dom = max(("tile_sort", "merge"), key=lambda c: kms[c])
    passes, merge_passes, merge_name = pass_counts(kernels, 2 * 12 * n)
    line = {
        "metric": "Gkeys/s and % HBM roofline, stable uint64+int32 pairs on 1 GB300", "value": n / (ms * 1e-3) / 1e9,
        "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64+i32", "data": "synthetic",
        "config": {"workload": f"stable pair sort, 2^{args.pairs_log2n} {args.pairs_dist} uint64 keys + int32 "
                               f"index payload, p={args.p} blocks", "n": n, "p": args.p,
                   "dist": args.pairs_dist, "tile_keys": 1 << args.pairs_tile_log2, "seed": SEED,
                   "l2": "inputs (12 B x n = 1.5 GiB at 2^27) larger than the 129 MB L2; no flush"},
        "roofline": {"bound": "hbm", "achieved": kernels[dom]["gbs"], "peak": peak, "unit": "GB/s",
                     "frac": kernels[dom]["gbs"] / peak, "traffic": None,
                     "kernel": (f"merge phase ({merge_name}: {merge_passes:g} passes per launch)"
                                if dom == "merge" else "tile sort"),
                     "peak_source": f"{peak_src} (copy bandwidth)", "passes_per_step": passes,
                     "end_to_end_frac": passes * 2 * 12 * n / (ms * 1e-3) / 1e9 / peak},
        "gpu_launches": int(sum(counts.values())), "clocks": clk, "kernels": kernels,
        "checked": "payload permutation, keys carried with payloads, nondecreasing, stable",
    }
    sorter.close()
    return line


# ---------------------------------------------------------------- batched workload

def run_batched(args):
    """Many int32 arrays of log-uniform length sorted by one graph-captured
    bs_sort_segmented, against one bs_sort_keys call per array."""
    import numpy as np
    import torch

    from paper_1105_6040_gb300 import abi, autotune
    from paper_1105_6040_gb300 import workloads as W

    rank, world, local = dist_env()
    if world != 1:
        raise SystemExit("the batched workload runs on one GPU")
    torch.cuda.set_device(local)
    hi = 1 << args.seg_hi_log2
    lens = W.loguniform_lengths(args.segments, args.seg_lo, hi, seed=SEED)
    off = W.offsets_from_lengths(lens)
    n = int(off[-1])
    if getattr(args, "device_gen", False):
        d_in = W.uniform_int32_torch(n, seed=SEED)  # the same bits, made on the GPU
    else:
        d_in = torch.from_numpy(W.uniform_int32(n, seed=SEED)).cuda()
    d_out = torch.empty_like(d_in)
    d_off = torch.from_numpy(off).cuda()
    sorter = abi.Sorter(local)
    t0 = time.perf_counter()
    cfg = autotune.tune(sorter, "segmented", d_in, offsets=d_off, max_seg_len=hi, repeats=1)
    tune_s = time.perf_counter() - t0
    graph = sorter.capture_segmented(d_in, d_off, d_out, max_seg_len=hi)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        graph.launch(stream)
    graph.sync()
    # every segment nondecreasing (segment starts may drop)
    starts = torch.zeros(n, dtype=torch.bool, device="cuda")
    starts[d_off[:-1][lens > 0].clamp(max=n - 1)] = True
    ok = (d_out[1:] >= d_out[:-1]) | starts[1:]
    assert bool(ok.all()), "batched output not sorted per segment"

    abi.bs_launch_stats(sorter.h, reset=True, with_bytes=False)
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        graph.launch(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_batched = e0.elapsed_time(e1) / args.steps

    # per-array baseline: one bs_sort_keys (p = 1) per array, same stream and buffers
    sp = stream.cuda_stream
    base_in, base_out = d_in.data_ptr(), d_out.data_ptr()

    def per_array_round():
        for i in range(args.segments):
            if lens[i]:
                abi.bs_sort_keys(sorter.h, base_in + 4 * int(off[i]), base_out + 4 * int(off[i]),
                                 int(lens[i]), "int32", 1, sp)

    abi.bs_launch_stats(sorter.h, reset=True, with_bytes=False)
    per_array_round()  # warm-up
    torch.cuda.synchronize()
    counts, _ = abi.bs_launch_stats(sorter.h, reset=True, with_bytes=False)
    per_array_launches = int(sum(counts.values()))
    e0.record(stream)
    for _ in range(args.per_array_rounds):
        per_array_round()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_per_array = e0.elapsed_time(e1) / args.per_array_rounds
    assert bool(((d_out[1:] >= d_out[:-1]) | starts[1:]).all())

    # per-kernel timing of one uncaptured run
    abi.bs_launch_stats(sorter.h, reset=True)
    abi.bs_set_option(sorter.h, "count_bytes", 1)
    sorter.set_timing(True)
    sorter.sort_segmented(d_in, d_off, kout=d_out, max_seg_len=hi)
    sorter.sync()
    sorter.set_timing(False)
    abi.bs_set_option(sorter.h, "count_bytes", 0)
    kms, kn = sorter.kernel_times()
    kcounts, kbytes = abi.bs_launch_stats(sorter.h, reset=True)
    peak, peak_src = load_peak()
    kernels = {c: {"launches": kn[c], "ms": kms[c],
                   "gbs": (kbytes[c] / (kms[c] * 1e-3) / 1e9) if kms[c] and kbytes[c] else None}
               for c in kms if kn[c]}
    graph.close()
    sorter.close()
    line = {
        "metric": f"Gkeys/s, batched segmented int32 sort ({args.segments} arrays, "
                  f"log-uniform lengths [{args.seg_lo}, 2^{args.seg_hi_log2}])",
        "value": n / (ms_batched * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_batched, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "batched segmented sort, one CUDA-graph replay per step",
                   "segments": args.segments, "total_keys": n, "seg_lo": args.seg_lo,
                   "seg_hi": hi, "mean_len": n / args.segments, "autotuned": cfg,
                   "autotune_s": tune_s, "seed": SEED},
        "per_array": {"value": n / (ms_per_array * 1e-3) / 1e9, "unit": UNIT,
                      "ms_per_step": ms_per_array, "launches_per_step": per_array_launches,
                      "api": "one bs_sort_keys(p=1) per array, same stream"},
        "speedup_vs_per_array": ms_per_array / ms_batched,
        "kernels_one_run": kernels, "clocks": clk,
        "roofline": {"bound": "hbm", "peak": peak, "unit": "GB/s",
                     "peak_source": f"{peak_src} (copy bandwidth)"},
    }
    return line


# ---------------------------------------------------------------- serving workload

def run_serving(args):
    """Poisson sort requests (lengths log-uniform [2^10, 2^26], int32 / float32
    50/50) served with continuous batching; p50/p99 latency and Gkeys/s."""
    import torch

    from paper_1105_6040_gb300 import serving as S

    rank, world, local = dist_env()
    if world != 1:
        raise SystemExit("the serving workload runs on one GPU")
    cfg = S.ServingConfig(rate=args.rate, duration=args.duration, streams=args.streams,
                          seed=SEED)
    clocks = ClockSampler(local)
    clocks.start()
    summary, reqs, ex = S.serve(cfg, device=local)
    clk = clocks.stop()
    ex.close()
    line = {
        "metric": "serving: p50/p99 latency (ms) and aggregate Gkeys/s, Poisson sort requests",
        "value": summary["gkeys_per_s"], "unit": UNIT, "n_gpus": 1, "steps": summary["requests"],
        "warmup": 0, "ms_per_step": summary["mean_ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "p50_ms": summary["p50_ms"], "p99_ms": summary["p99_ms"],
        "config": {"workload": "serving loop with continuous batching",
                   **{k: v for k, v in dataclasses_asdict(cfg).items() if k != "keep_results"}},
        "serving": summary, "clocks": clk,
        "offered_gkeys_per_s": sum(r.n for r in reqs) / cfg.duration / 1e9,
    }
    return line


# ---------------------------------------------------------------- p sweep (Table 1 analogue)

def run_psweep(args):
    """Time against the number of blocks p, the GPU analogue of the paper's
    Exp. 1 / Table 1: for each key distribution, the pairwise tree (the
    default path: 8192-key tiles, the persistent merge) at p = 1 .. 4096 and
    Fig. 1's odd-even compare-split schedule at p = 1 .. 64, with the time of
    each kernel class and the passes per sort."""
    import torch

    from paper_1105_6040_gb300 import abi
    from paper_1105_6040_gb300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    n = 1 << args.log2n
    out = None
    rows = []
    stream = torch.cuda.current_stream()
    dists = args.dists.split(",") if args.dists else [args.dist]
    for dist in dists:
        x = W.int32_keys_torch(dist, n, seed=SEED)
        out = torch.empty_like(x)
        for sched in ("tree", "oddeven"):
            ps = [1 << i for i in range(13)] if sched == "tree" else [1, 2, 4, 8, 16, 32, 64]
            s = abi.Sorter(local, tile_log2=args.tile_log2)
            abi.bs_set_option(s.h, "merge_schedule", sched)
            for p in ps:
                for _ in range(2):
                    s.sort_keys(x, out=out, p=p)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                reps = max(2, min(args.steps, 10))
                e0.record(stream)
                for _ in range(reps):
                    s.sort_keys(x, out=out, p=p)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
                # one more sort with per-launch events and counted bytes
                s.stats(reset=True)
                abi.bs_set_option(s.h, "count_bytes", 1)
                s.set_timing(True)
                s.sort_keys(x, out=out, p=p)
                s.sync()
                s.set_timing(False)
                abi.bs_set_option(s.h, "count_bytes", 0)
                kms, kn = s.kernel_times()
                counts, byts = s.stats(reset=True)
                rows.append({"dist": dist, "schedule": sched, "p": p, "ms": ms,
                             "gkeys_per_s": n / (ms * 1e-3) / 1e9,
                             "passes": (byts["tile_sort"] + byts["merge"]) / (2 * 4 * n),
                             "launches": int(sum(counts.values())),
                             "kernel_ms": {k: round(v, 4) for k, v in kms.items() if kn[k]}})
            assert bool((out[1:] >= out[:-1]).all())
            s.close()
        del x, out
        torch.cuda.empty_cache()
    line = {"metric": f"time vs p, 2^{args.log2n} int32 keys (Table 1 analogue)",
            "value": min(r["ms"] for r in rows), "unit": "ms", "n_gpus": 1,
            "higher_is_better": False, "data": "synthetic", "rows": rows,
            "config": {**config(args), "dists": dists}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- local sorts (Figs. 2-4)

def run_localsort(args):
    """Sort-phase tile sorts after the paper's three local sorts (merge,
    bubble, quick) on one input: tile-sort kernel time and whole-sort time."""
    import torch

    from paper_1105_6040_gb300 import abi

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    args.tile_log2, args.merge_tile_log2 = 12, 0  # the 4096-key tile every row uses (for config())
    n = 1 << args.log2n
    x = torch.from_numpy(make_keys(args, 0)).cuda()
    out = torch.empty_like(x)
    rows = []
    for ls in ("merge", "quick", "bubble"):
        s = abi.Sorter(local, tile_log2=12)  # the 4096-key tile every row of this table uses
        abi.bs_set_option(s.h, "local_sort", ls)
        s.sort_keys(x, out=out, p=args.p)
        s.sync()
        s.stats(reset=True)
        s.set_timing(True)
        reps = 3
        for _ in range(reps):
            s.sort_keys(x, out=out, p=args.p)
        s.sync()
        s.set_timing(False)
        kms, kn = s.kernel_times()
        total = sum(kms.values()) / reps
        rows.append({"local_sort": ls, "tile_sort_ms": kms["tile_sort"] / max(1, kn["tile_sort"]),
                     "sort_ms": total, "gkeys_per_s": n / (total * 1e-3) / 1e9})
        assert bool((out[1:] >= out[:-1]).all())
        s.close()
    line = {"metric": f"sort-phase tile sorts (Figs. 2-4), 2^{args.log2n} {args.dist} int32, p={args.p}",
            "value": rows[0]["sort_ms"], "unit": "ms", "n_gpus": 1, "higher_is_better": False,
            "data": "synthetic", "rows": rows, "config": config(args)}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- memory experiment

def run_memory(args):
    """Device memory against n with two blocks (the paper's Exp. 2 / Table 2
    analogue): the scratch the library asks for (bs_workspace_bytes) and the
    device memory one sort actually took (cudaMemGetInfo before and after)."""
    import torch

    from paper_1105_6040_gb300 import abi
    from paper_1105_6040_gb300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    rows = []
    for n in [int(2.5e6 + 5e5 * i) for i in range(6)]:  # Table 2's sizes for merge / quick sort
        ws = abi.bs_workspace_bytes(n, 2, "int32")
        x = torch.from_numpy(W.uniform_int32(n, seed=SEED)).cuda()
        out = torch.empty_like(x)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        s = abi.Sorter(local)
        s.sort_keys(x, out=out, p=2)
        s.sync()
        free1, _ = torch.cuda.mem_get_info()
        s.close()
        rows.append({"n": n, "workspace_bytes": ws, "device_bytes_taken": free0 - free1,
                     "in_out_bytes": 8 * n,
                     "bytes_per_item_total": (ws + 8 * n) / n})
    line = {"metric": "device memory vs n, int32 keys, p=2 (Table 2 analogue)", "value": rows[-1]["bytes_per_item_total"],
            "unit": "bytes/item", "n_gpus": 1, "higher_is_better": False, "data": "synthetic",
            "rows": rows,
            "paper_context": {"merge_sort_bytes_per_item": 83.9, "quick_sort_bytes_per_item": 13.7,
                              "bubble_sort_bytes_per_item": 11.8, "note": "2011 Windows process memory"}}
    print(json.dumps(line), flush=True)
    return 0


def dataclasses_asdict(x):
    import dataclasses
    return dataclasses.asdict(x)


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload in ("batched", "serving", "pairs"):
        fn = {"batched": run_batched, "serving": run_serving, "pairs": run_pairs}[args.workload]
        print(json.dumps(fn(args)), flush=True)
        return 0
    if args.workload == "memory":
        return run_memory(args)
    if args.workload == "psweep":
        return run_psweep(args)
    if args.workload == "localsort":
        return run_localsort(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
