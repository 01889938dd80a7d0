"""Continuous-batching policy of the serving loop, on the CPU with a fake
executor and a fake clock (no GPU)."""
import numpy as np

from paper_1105_6040_gb300 import serving as S


class FakeClock:
    def __init__(self, dt=50e-6):
        self.t, self.dt = 0.0, dt

    def __call__(self):
        self.t += self.dt
        return self.t


class FakeExecutor:
    """Slots that finish a batch after 1 ns per key plus 20 us."""

    def __init__(self, slots, clock):
        self.slots = [None] * slots
        self.clock = clock
        self.log = []            # (launch time, batch)
        self.max_concurrent = 0

    def start(self, clock):
        return clock()

    def free_slots(self):
        return [i for i, s in enumerate(self.slots) if s is None]

    @staticmethod
    def bytes_for(batch):
        return 8 * sum(r.n for r in batch)

    def launch(self, slot, batch):
        now = self.clock.t
        self.log.append((now, list(batch)))
        self.slots[slot] = (batch, now + 20e-6 + 1e-9 * sum(r.n for r in batch))
        self.max_concurrent = max(self.max_concurrent, sum(s is not None for s in self.slots))

    def poll(self):
        out = []
        for i, s in enumerate(self.slots):
            if s is not None and s[1] <= self.clock.t:
                out.append((s[0], s[1]))
                self.slots[i] = None
        return out

    def idle(self):
        pass


def run(cfg, cap, slots=4):
    clock = FakeClock()
    ex = FakeExecutor(slots, clock)
    reqs = S.make_requests(cfg)
    sched = S.Scheduler(cfg, ex, cap)
    summary = sched.run(reqs, clock=clock)
    return summary, reqs, ex, sched


CFG = S.ServingConfig(rate=2000, duration=0.5, lo=1 << 10, hi=1 << 20, small_max=1 << 14,
                      batch_max_keys=1 << 18, batch_max_reqs=64, pool_keys=1 << 21)


def test_every_request_completes_after_it_arrives():
    summary, reqs, ex, _ = run(CFG, cap=1 << 40)
    assert summary["requests"] == len(reqs) > 500
    for r in reqs:
        assert r.arrival <= r.launched <= r.done
    assert summary["p50_ms"] <= summary["p99_ms"] <= summary["max_ms"]


def test_batches_are_small_same_dtype_or_single_large():
    _, _, ex, _ = run(CFG, cap=1 << 40)
    multi = 0
    for _, batch in ex.log:
        if len(batch) > 1:
            multi += 1
            assert all(r.n <= CFG.small_max for r in batch)
            assert len({r.dtype for r in batch}) == 1
            assert sum(r.n for r in batch) <= CFG.batch_max_keys or len(batch) == 1
            assert len(batch) <= CFG.batch_max_reqs
    assert multi > 0  # continuous batching did happen


def test_work_overlaps_on_several_slots():
    _, _, ex, _ = run(CFG, cap=1 << 40, slots=4)
    assert ex.max_concurrent > 1


def test_admission_cap_holds_and_defers():
    cap = 8 * (1 << 20)  # one large request at most
    summary, reqs, ex, sched = run(CFG, cap=cap)
    assert summary["requests"] == len(reqs)
    assert sched.peak_bytes <= cap or all(len(b) == 1 for _, b in ex.log)
    assert sched.deferrals > 0


def test_requests_are_reproducible_from_the_seed():
    a, b = S.make_requests(CFG), S.make_requests(CFG)
    assert [(r.arrival, r.n, r.dtype, r.src) for r in a] == [(r.arrival, r.n, r.dtype, r.src) for r in b]
    lens = np.array([r.n for r in a])
    assert lens.min() >= CFG.lo and lens.max() <= CFG.hi
    assert all(0 <= r.src <= CFG.pool_keys - r.n for r in a)
    assert {r.dtype for r in a} == {"int32", "float32"}
