"""Serving loop: sort requests of mixed sizes and dtypes with continuous batching.

Requests arrive over time (a Poisson process).  Their keys are already
resident on the GPU: every request is a slice of a device pool of its dtype.
A single-threaded scheduler runs the loop:

* arrivals whose time has come join the pending queue (FIFO);
* whenever an execution slot (a CUDA stream with its own library handle) is
  free, the head of the queue is launched: a large request alone
  (bs_sort_keys), a small one together with every other pending small request
  of the same dtype, up to a key and request budget, as ONE gathered
  segmented sort (bs_sort_segmented_gather: each segment reads its keys from
  its own place in the pool, so no gather copy is needed);
* every slot's library handle reserves its scratch once, at start-up
  (bs_reserve_workspace: enough for the largest request or batch it may
  run), so a launch allocates only its output; a launch is admitted only
  while the output bytes held by work in flight stay under the memory cap (by
  default 80% of the HBM still free once pools and scratch are in place);
  otherwise it waits for running work to finish (a launch with nothing in
  flight is always admitted, so one request over the cap cannot stall the
  loop);
* completions are detected by CUDA events; a request's latency is the time
  from its arrival to the end of its GPU work (both measured from one common
  origin: a start event recorded when the loop starts).

Work on different slots overlaps on the device.  Sorting is exact, so a
request's result is the same alone and in the mix, bit for bit.

``Scheduler`` holds the policy and talks to an executor through four calls
(free_slots, bytes_for, launch, poll), so the policy is testable without a GPU
(see FakeExecutor in the tests).
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import workloads as W

DTYPE_NAMES = ("int32", "float32")


@dataclasses.dataclass
class ServingConfig:
    rate: float = 2000.0          # requests per second (Poisson)
    duration: float = 60.0        # seconds of arrivals
    lo: int = 1 << 10             # request lengths: log-uniform in [lo, hi]
    hi: int = 1 << 26
    small_max: int = 1 << 16      # requests up to this many keys are batched
    batch_max_keys: int = 1 << 22
    batch_max_reqs: int = 1024
    streams: int = 4              # execution slots
    mem_frac: float = 0.8         # admission cap: fraction of free HBM at start
    mem_cap_bytes: int = 0        # explicit cap (overrides mem_frac when > 0)
    pool_keys: int = 1 << 27      # keys per dtype pool (>= hi)
    seed: int = W.DEFAULT_SEED
    keep_results: bool = False    # keep every output (for verification)


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float                # seconds from the loop start
    n: int
    dtype: str
    src: int                      # offset of its keys in the pool of its dtype
    launched: float = -1.0
    done: float = -1.0
    batch: int = -1
    result: object = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def make_requests(cfg: ServingConfig) -> list[Request]:
    t = W.poisson_arrivals(cfg.rate, cfg.duration, seed=cfg.seed)
    m = t.size
    lens = W.loguniform_lengths(m, cfg.lo, cfg.hi, seed=cfg.seed ^ 0x1)
    kinds = W.coin(m, seed=cfg.seed ^ 0x2)
    span = np.maximum(cfg.pool_keys - lens, 0).astype(np.uint64) + np.uint64(1)
    src = (W.splitmix64(cfg.seed ^ 0x3, 0, m) % span).astype(np.int64)
    return [Request(i, float(t[i]), int(lens[i]), DTYPE_NAMES[int(kinds[i])], int(src[i]))
            for i in range(m)]


class Scheduler:
    """Continuous batching with memory admission (policy only)."""

    def __init__(self, cfg: ServingConfig, executor, mem_cap_bytes: int):
        self.cfg = cfg
        self.ex = executor
        self.cap = int(mem_cap_bytes)
        self.in_flight_bytes = 0
        self.peak_bytes = 0
        self.deferrals = 0
        self.batches = 0
        self.batch_sizes: list[int] = []

    def _form_batch(self, pending: list[Request]) -> list[Request]:
        head = pending[0]
        if head.n > self.cfg.small_max:
            return [head]
        batch, keys = [], 0
        for r in pending:
            if r.n > self.cfg.small_max or r.dtype != head.dtype:
                continue
            if batch and (keys + r.n > self.cfg.batch_max_keys or len(batch) >= self.cfg.batch_max_reqs):
                break
            batch.append(r)
            keys += r.n
        return batch

    def run(self, requests: list[Request], clock=time.perf_counter) -> dict:
        order = sorted(requests, key=lambda r: r.arrival)
        pending: list[Request] = []
        nxt, finished = 0, 0
        t0 = self.ex.start(clock)
        while finished < len(order):
            now = clock() - t0
            while nxt < len(order) and order[nxt].arrival <= now:
                pending.append(order[nxt])
                nxt += 1
            for batch, done in self.ex.poll():
                for r in batch:
                    r.done = done
                self.in_flight_bytes -= self.ex.bytes_for(batch)
                finished += len(batch)
            launched = False
            while pending:
                slots = self.ex.free_slots()
                if not slots:
                    break
                batch = self._form_batch(pending)
                need = self.ex.bytes_for(batch)
                if self.in_flight_bytes + need > self.cap and self.in_flight_bytes > 0:
                    self.deferrals += 1
                    break
                ids = {r.rid for r in batch}
                pending = [r for r in pending if r.rid not in ids]
                for r in batch:
                    r.launched = now
                    r.batch = self.batches
                self.ex.launch(slots[0], batch)
                self.in_flight_bytes += need
                self.peak_bytes = max(self.peak_bytes, self.in_flight_bytes)
                self.batches += 1
                self.batch_sizes.append(len(batch))
                launched = True
            if not launched:
                self.ex.idle()
        return summarize(order, self)


def summarize(reqs: list[Request], sched: Scheduler) -> dict:
    lat = np.array([r.latency for r in reqs]) * 1e3
    keys = sum(r.n for r in reqs)
    span = max(r.done for r in reqs) - min(r.arrival for r in reqs)
    return {
        "requests": len(reqs), "keys": keys, "seconds": span,
        "gkeys_per_s": keys / span / 1e9 if span > 0 else None,
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
        "batches": sched.batches,
        "mean_batch_requests": float(np.mean(sched.batch_sizes)) if sched.batch_sizes else 0.0,
        "deferrals": sched.deferrals, "peak_in_flight_bytes": sched.peak_bytes,
        "mem_cap_bytes": sched.cap,
        "reserved_scratch_bytes": int(getattr(sched.ex, "reserved_bytes", 0)),
    }


class GpuExecutor:
    """Executes batches on CUDA streams, one library handle per stream."""

    def __init__(self, cfg: ServingConfig, device: int = 0):
        import torch

        from .abi import Sorter, bs_reserve_workspace
        self.torch = torch
        self.cfg = cfg
        self.dev = torch.device("cuda", device)
        torch.cuda.set_device(self.dev)
        n = cfg.pool_keys
        self.pools = {
            "int32": torch.from_numpy(W.uniform_int32(n, seed=cfg.seed ^ 0x10)).to(self.dev),
            "float32": torch.from_numpy(W.normal_float32_edges(n, seed=cfg.seed ^ 0x11)).to(self.dev),
        }
        self.slots = []
        self.reserved_bytes = 0
        # the largest call a slot makes: one request of up to hi keys, or a
        # batch of up to batch_max_keys keys in up to batch_max_reqs segments
        res_n = max(cfg.hi, cfg.batch_max_keys)
        res_s = max(1, cfg.batch_max_reqs)
        for _ in range(cfg.streams):
            sorter = Sorter(device)
            self.reserved_bytes += bs_reserve_workspace(sorter.h, res_n, res_s, "int32")
            self.slots.append({"stream": torch.cuda.Stream(self.dev), "sorter": sorter, "busy": None})
        self.start_event = None
        self._warm_up()

    def _warm_up(self):
        """Run each slot once through every path a request can take (a lone
        request of each size class, a gathered batch), so that no request
        pays for loading the library's kernels on their first use."""
        t, cfg = self.torch, self.cfg
        pool = self.pools["int32"]
        sizes, n = [], max(cfg.lo, 1)
        while n <= min(cfg.hi, pool.numel()):
            sizes.append(n)
            n *= 4
        for slot in self.slots:
            st, sorter = slot["stream"], slot["sorter"]
            with t.cuda.stream(st):
                for n in sizes:
                    sorter.sort_keys(pool[:n], p=1, stream=st)
                k = min(cfg.batch_max_reqs, 8)
                lens = np.full(k, max(1, min(cfg.small_max, cfg.batch_max_keys // k)), dtype=np.int64)
                off = W.offsets_from_lengths(lens)
                src = np.zeros(k, dtype=np.int64)
                sorter.sort_gathered(pool, t.from_numpy(src).to(self.dev), t.from_numpy(off).to(self.dev),
                                     max_seg_len=int(lens.max()), stream=st)
            sorter.sync()
        t.cuda.synchronize()

    # -- executor interface
    def start(self, clock):
        t = self.torch
        t.cuda.synchronize()
        self.start_event = t.cuda.Event(enable_timing=True)
        self.start_event.record()
        self.start_event.synchronize()
        return clock()

    def free_slots(self):
        return [i for i, s in enumerate(self.slots) if s["busy"] is None]

    @staticmethod
    def bytes_for(batch) -> int:
        # what a launch allocates: its output (4-byte keys) and, for a batch,
        # the segment offsets and sources (the handles' scratch is reserved)
        keys = sum(r.n for r in batch)
        return 4 * keys + (16 * (len(batch) + 1) if len(batch) > 1 else 0)

    def scratch_bytes(self) -> int:
        """The slots' handles' scratch now (unchanged from the reservation
        unless a call needed more)."""
        from .abi import bs_reserve_workspace
        return sum(bs_reserve_workspace(s["sorter"].h, 0, 1, "int32") for s in self.slots)

    def launch(self, slot_id: int, batch: list[Request]):
        t = self.torch
        slot = self.slots[slot_id]
        st, sorter = slot["stream"], slot["sorter"]
        pool = self.pools[batch[0].dtype]
        with t.cuda.stream(st):
            if len(batch) == 1 and batch[0].n > self.cfg.small_max:
                r = batch[0]
                out = t.empty(r.n, dtype=pool.dtype, device=self.dev)
                sorter.sort_keys(pool[r.src:r.src + r.n], out=out, p=1, stream=st)
                views = [out]
            else:
                lens = np.array([r.n for r in batch], dtype=np.int64)
                off = W.offsets_from_lengths(lens)
                src = np.array([r.src for r in batch], dtype=np.int64)
                meta = t.from_numpy(np.concatenate([off, src])).pin_memory().to(self.dev, non_blocking=True)
                d_off, d_src = meta[:off.size], meta[off.size:]
                out = t.empty(int(off[-1]), dtype=pool.dtype, device=self.dev)
                sorter.sort_gathered(pool, d_src, d_off, kout=out, max_seg_len=int(lens.max()),
                                     stream=st)
                views = [out[off[i]:off[i + 1]] for i in range(len(batch))]
            ev = t.cuda.Event(enable_timing=True)
            ev.record(st)
        slot["busy"] = (batch, views, ev)

    def poll(self):
        done = []
        for s in self.slots:
            if s["busy"] is None:
                continue
            batch, views, ev = s["busy"]
            if ev.query():
                t_done = self.start_event.elapsed_time(ev) * 1e-3
                if self.cfg.keep_results:
                    for r, v in zip(batch, views):
                        r.result = v
                s["busy"] = None
                done.append((batch, t_done))
        return done

    def idle(self):
        time.sleep(20e-6)

    def check(self):
        for s in self.slots:
            s["sorter"].sync()

    def close(self):
        for s in self.slots:
            s["sorter"].close()


def default_mem_cap(cfg: ServingConfig) -> int:
    if cfg.mem_cap_bytes > 0:
        return cfg.mem_cap_bytes
    import torch
    free, _ = torch.cuda.mem_get_info()
    return int(cfg.mem_frac * free)


def serve(cfg: ServingConfig, device: int = 0):
    """Run one serving session on the GPU; returns (summary, requests, executor)."""
    ex = GpuExecutor(cfg, device)
    cap = default_mem_cap(cfg)
    reqs = make_requests(cfg)
    sched = Scheduler(cfg, ex, cap)
    summary = sched.run(reqs)
    ex.check()
    return summary, reqs, ex
