"""Admission policy of the gradient server on the host (no GPU): FIFO by device footprint and slots,
the batch lane's run limit, and large grids one at a time with smaller requests allowed to overtake one
that waits for a running large grid (large grids stay in FIFO order among themselves)."""
import collections

import pytest

serve = pytest.importorskip("paper_2305_00234_gb300.serve")


class FakeRequest:
    def __init__(self, n, precision=32):
        self.n = n
        self.desc = {"nx": n, "ny": n, "nz": n, "precision": precision}

    def cells(self):
        return self.n ** 3


def server(budget=100, slots=4, batch_max_cells=0, exclusive_cells=128 ** 3):
    """A GradientServer with its admission state only (no device, no dispatcher thread)."""
    s = object.__new__(serve.GradientServer)
    s.hbm_budget = budget
    s.max_slots = slots
    s.batch_max_cells = batch_max_cells
    s.exclusive_cells = exclusive_cells
    s.exclusive_running = 0
    s.waiting = collections.deque()
    s.in_use = 0
    s.active = 0
    s.batch_pending = 0
    s.in_batch = {}
    s.peak_active = 0
    s.peak_in_use = 0
    return s


def queue(s, *reqs):
    for r, fp in reqs:
        s.waiting.append((r, fp, object()))


def admit_all(s):
    out = []
    while s._can_admit():
        req, fp, fut, t = s._admit_one()
        out.append(req)
    return out


def test_fifo_stops_at_the_first_request_that_does_not_fit():
    s = server(budget=100)
    a, b, c = FakeRequest(48), FakeRequest(64), FakeRequest(48)
    queue(s, (a, 60), (b, 50), (c, 10))
    assert admit_all(s) == [a]                  # b does not fit; c may not pass it
    assert s.in_use == 60 and s.active == 1
    s.in_use -= 60                              # a finishes
    s.active -= 1
    assert admit_all(s) == [b, c]


def test_slots_bound_the_requests_on_the_device():
    s = server(budget=10 ** 9, slots=2)
    reqs = [FakeRequest(48) for _ in range(4)]
    queue(s, *[(r, 1) for r in reqs])
    assert admit_all(s) == reqs[:2]
    assert s.peak_active == 2


def test_large_grids_one_at_a_time_and_small_ones_overtake():
    s = server(budget=10 ** 9, slots=8, exclusive_cells=128 ** 3)
    big1, big2, small, big3, small2 = (FakeRequest(192), FakeRequest(128), FakeRequest(64), FakeRequest(192),
                                       FakeRequest(96))
    queue(s, (big1, 1), (big2, 1), (small, 1), (big3, 1), (small2, 1))
    got = admit_all(s)
    assert got == [big1, small, small2]         # big2 waits for big1; the small ones pass it
    assert [r for r, _, _ in s.waiting] == [big2, big3]
    assert s.exclusive_running == 1
    # big1 finishes: big2 (first of the waiting large grids) starts, big3 keeps waiting
    s.exclusive_running -= 1
    s.active -= 1
    assert admit_all(s) == [big2]
    assert [r for r, _, _ in s.waiting] == [big3]


def test_strict_fifo_without_the_large_grid_rule():
    s = server(budget=10 ** 9, slots=8, exclusive_cells=None)
    reqs = [FakeRequest(192), FakeRequest(192), FakeRequest(48)]
    queue(s, *[(r, 1) for r in reqs])
    assert admit_all(s) == reqs                 # large grids side by side when the rule is off


def test_batch_lane_run_limit_and_lane_choice():
    s = server(budget=10 ** 9, slots=32, batch_max_cells=64 ** 3, exclusive_cells=None)
    small = [FakeRequest(48) for _ in range(serve.N.MAX_BATCH + 2)]
    fp64 = FakeRequest(48, precision=64)
    assert s._batch_lane(small[0]) and not s._batch_lane(FakeRequest(96)) and not s._batch_lane(fp64)
    queue(s, *[(r, 1) for r in small])
    got = admit_all(s)
    assert len(got) == serve.N.MAX_BATCH       # the batch lane holds at most MAX_BATCH runs
    assert s.batch_pending == serve.N.MAX_BATCH
