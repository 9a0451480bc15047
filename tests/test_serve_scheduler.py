"""Host logic of the serving loop (no GPU): admission by HBM footprint,
slots, FIFO with skip-ahead, rejection reasons, simulated completion."""
import heapq

import numpy as np

from paper_1003_2022_gb300.serve import Scheduler, footprint_bytes


def _simulate(arrivals, sizes, durations, slots, budget, Ns=None):
    """Discrete-event run of the scheduler; returns admit/done times and peak usage."""
    sch = Scheduler(slots, budget)
    events = [(t, 0, i) for i, t in enumerate(arrivals)]  # (time, kind 0 arrival / 1 done, rid)
    heapq.heapify(events)
    admit, done, rejected = {}, {}, {}
    while events:
        t, kind, rid = heapq.heappop(events)
        if kind == 0:
            why = sch.offer(rid, sizes[rid], (Ns or [4] * len(sizes))[rid])
            if why:
                rejected[rid] = why
        else:
            sch.complete(rid)
            done[rid] = t
        assert sch.used() <= budget
        assert len(sch.inflight) <= slots
        for r, slot in sch.admit():
            admit[r] = t
            heapq.heappush(events, (t + durations[r], 1, r))
    return admit, done, rejected, sch.peak_bytes


def test_budget_and_slots_never_exceeded_and_all_finish():
    rng = np.random.default_rng(0)
    n = 300
    arrivals = np.cumsum(rng.exponential(0.01, n))
    sizes = rng.integers(1, 40, n) * (1 << 20)
    durations = sizes / (1 << 30) + 0.001
    admit, done, rejected, peak = _simulate(arrivals, sizes, durations, slots=4, budget=100 << 20)
    assert not rejected
    assert len(done) == n
    assert peak <= 100 << 20
    for r in range(n):
        assert admit[r] >= arrivals[r] and done[r] >= admit[r]


def test_skip_ahead_lets_small_requests_pass_a_blocked_large_one():
    # one long request holds 70 of 100 units; a 50-unit request must wait, a 10-unit one passes it
    arrivals = [0.0, 0.1, 0.2]
    sizes = [70, 50, 10]
    durations = [10.0, 1.0, 1.0]
    admit, done, rejected, _ = _simulate(arrivals, sizes, durations, slots=4, budget=100)
    assert admit[2] < admit[1]
    assert admit[1] == done[0]


def test_continuous_admission_while_others_run():
    # two slots: the third request starts as soon as the first finishes, not after a batch drains
    arrivals = [0.0, 0.0, 0.05]
    sizes = [1, 1, 1]
    durations = [0.1, 1.0, 0.1]
    admit, done, _, _ = _simulate(arrivals, sizes, durations, slots=2, budget=10)
    assert admit[2] == done[0] and admit[2] < done[1]


def test_rejections_have_reasons():
    sch = Scheduler(2, 1000)
    assert "budget" in sch.offer(0, 5000, 4)
    assert sch.offer(1, 10, 6) is None
    assert "N=5" in sch.offer(2, 10, 5)
    assert sch.offer(2, 10, 4) is None


def test_footprint_grows_with_size_channels_and_sigma():
    f1 = footprint_bytes(1, 256, 256, 4, 2.0)
    assert footprint_bytes(3, 256, 256, 4, 2.0) > 2.5 * f1
    assert footprint_bytes(1, 512, 512, 4, 2.0) > 3.5 * f1
    assert footprint_bytes(1, 256, 256, 4, 40.0) > f1
    assert footprint_bytes(1, 256, 256, 1, 2.0) < f1
    # six directions: FP64 scales and lattice windows, growing with the footprint
    g1 = footprint_bytes(1, 256, 256, 4, 2.0, 6)
    assert g1 > 48 * 256 * 256 and footprint_bytes(1, 256, 256, 4, 20.0, 6) > 4 * g1
    # two window buffers of at most 8 GiB each, plus scales and the request's own tensors
    assert footprint_bytes(3, 4096, 4096, 4, 48.0, 6) < 2 * (8 << 30) + 4096 * 4096 * (48 + 40)


def test_cancel_only_queued_requests():
    s = Scheduler(slots=1, budget_bytes=100)
    assert s.offer(1, 10, 4) is None and s.offer(2, 10, 4) is None and s.offer(3, 10, 4) is None
    assert s.admit() == [(1, 0)]
    assert s.cancel(2) is True          # queued: withdrawn
    assert s.cancel(2) is False         # already gone
    assert s.cancel(1) is False         # in flight: runs to completion
    assert s.cancel(99) is False        # unknown
    s.complete(1)
    assert s.admit() == [(3, 0)]
