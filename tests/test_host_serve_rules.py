"""The serving loop's host-side rules, checked on the CPU with stand-in
requests and events (no GPU): the admission rule that keeps a lone arrival
waiting while a request is in flight, and the batch rule that takes only
finished sorts from a short queue."""

import dataclasses

from paper_2509_25626_gb300.serve import batch_size, may_admit, poisson_requests


@dataclasses.dataclass
class Req:
    arrival: float


class Ev:
    def __init__(self, done: bool):
        self.done = done
        self.queries = 0

    def query(self) -> bool:
        self.queries += 1
        return self.done


def test_admission_waits_for_overlap_min_arrivals_while_busy():
    pending = [Req(0.10), Req(0.20), Req(0.30)]
    # idle GPU: whatever has arrived is admitted
    assert may_admit(pending, 0.15, in_flight=False, realtime=True, overlap_min=2)
    # busy: one arrival waits, two start
    assert not may_admit(pending, 0.15, in_flight=True, realtime=True, overlap_min=2)
    assert may_admit(pending, 0.25, in_flight=True, realtime=True, overlap_min=2)
    assert not may_admit(pending, 0.25, in_flight=True, realtime=True, overlap_min=3)
    assert may_admit(pending, 0.35, in_flight=True, realtime=True, overlap_min=3)
    # nothing arrived yet
    assert not may_admit(pending, 0.05, in_flight=True, realtime=True, overlap_min=2)
    # overlap_min 1 (always overlap) and saturation runs admit at once
    assert may_admit(pending, 0.15, in_flight=True, realtime=True, overlap_min=1)
    assert may_admit(pending, 0.0, in_flight=True, realtime=False, overlap_min=4)
    assert may_admit([], 1.0, in_flight=True, realtime=True, overlap_min=1)


def test_batch_takes_finished_sorts_from_a_short_queue():
    ev = lambda *d: [Ev(x) for x in d]
    # the oldest always goes, even unfinished; then the leading finished ones
    assert batch_size(ev(False, True, True), 16, 3) == 3
    assert batch_size(ev(True, False, True), 16, 3) == 1
    assert batch_size(ev(False), 16, 3) == 1
    assert batch_size(ev(True, True, False), 16, 3) == 2
    # a long queue is batched whole, up to max_batch, without queries
    long_q = ev(*([False] * 5))
    assert batch_size(long_q, 16, 3) == 5 and all(e.queries == 0 for e in long_q)
    assert batch_size(ev(*([True] * 20)), 16, 0) == 16
    assert batch_size(ev(False, False), 1, 3) == 1
    assert batch_size([], 16, 3) == 0
    # ready_only off (0): everything up to max_batch
    assert batch_size(ev(False, False, False), 16, 0) == 3


def test_poisson_requests_are_ordered_and_within_duration():
    reqs = poisson_requests(500.0, 0.2, ["a", "b"], [(64, 48), (96, 64)], lambda u, w, h: (u, w, h), seed=1)
    assert 50 < len(reqs) < 160
    t = [r.arrival for r in reqs]
    assert t == sorted(t) and 0.0 < t[0] and t[-1] <= 0.2
    assert {r.scene for r in reqs} == {"a", "b"}
    assert [r.rid for r in reqs] == list(range(len(reqs)))
