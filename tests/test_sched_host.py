"""Admission scheduler of the serving loop (occ_sched_*): host-only policy tests.

FIFO admission under a byte budget, no overtaking, batch size and in-flight limits, queue
limit, deadlines, drain, and a randomized run against a plain Python model of the policy.
"""
import random
import threading

import pytest

from paper_2607_23122_gb300 import _native as N
from paper_2607_23122_gb300.occ import Scheduler

OK, INVALID, OOM, BUSY = 0, 1, 3, 7


def test_invalid_configs_are_refused():
    for kw in (dict(budget_bytes=0), dict(budget_bytes=10, max_views_per_batch=0),
               dict(budget_bytes=10, max_views_per_batch=257), dict(budget_bytes=10, max_inflight=0),
               dict(budget_bytes=10, max_inflight=17), dict(budget_bytes=10, max_queued=0)):
        with pytest.raises(Exception):
            Scheduler(**kw)


def test_fifo_admission_within_budget():
    s = Scheduler(100, max_views_per_batch=8, max_inflight=2)
    for i in range(1, 6):
        assert s.submit(i, 30, 0) == OK
    slot, ids, exp = s.next(1)
    assert (slot, ids, exp) == (0, [1, 2, 3], [])
    assert s.next(2) == (-1, [], [])          # 90 + 30 > 100 although slot 1 is free
    st = s.stats()
    assert st["reserved_bytes"] == 90 and st["inflight_batches"] == 1 and st["queued"] == 2
    assert s.complete(0) == OK
    slot, ids, _ = s.next(3)
    assert ids == [4, 5] and slot in (0, 1)
    assert s.complete(slot) == OK
    st = s.stats()
    assert st["reserved_bytes"] == 0 and st["peak_reserved_bytes"] == 90
    assert st["admitted"] == 5 and st["completed_batches"] == 2


def test_no_overtaking_of_a_large_request():
    s = Scheduler(100, max_inflight=4)
    s.submit(1, 60, 0)
    s.submit(2, 60, 0)
    s.submit(3, 10, 0)
    slot, ids, _ = s.next(1)
    assert ids == [1]                          # 2 does not fit; 3 fits but may not overtake
    assert s.next(2)[1] == []
    s.complete(slot)
    assert s.next(3)[1] == [2, 3]


def test_batch_size_and_inflight_limits():
    s = Scheduler(1000, max_views_per_batch=2, max_inflight=2)
    for i in range(1, 8):
        s.submit(i, 1, 0)
    a = s.next(1)
    b = s.next(1)
    assert a[1] == [1, 2] and b[1] == [3, 4] and {a[0], b[0]} == {0, 1}
    assert s.next(1) == (-1, [], [])          # both slots busy
    s.complete(b[0])
    c = s.next(2)
    assert c == (b[0], [5, 6], [])
    assert s.complete(5) == INVALID and s.complete(-1) == INVALID
    s.complete(a[0])
    assert s.complete(a[0]) == INVALID        # already free


def test_refusals():
    s = Scheduler(100, max_queued=2)
    assert s.submit(1, 0, 0) == INVALID
    assert s.submit(1, -5, 0) == INVALID
    assert s.submit(1, 101, 0) == OOM
    assert s.submit(1, 100, 0) == OK
    assert s.submit(1, 10, 0) == INVALID       # id still queued
    assert s.submit(2, 10, 0) == OK
    assert s.submit(3, 10, 0) == BUSY          # queue full
    slot, ids, _ = s.next(0)
    assert ids == [1]
    assert s.submit(1, 10, 0) == INVALID       # id still running
    assert s.submit(3, 10, 0) == OK
    s.complete(slot)
    assert s.next(0)[1] == [2, 3]
    assert s.submit(1, 10, 0) == OK            # finished ids may be reused
    st = s.stats()
    assert st["refused"] == 6 and st["submitted"] == 10


def test_deadlines_expire_queued_requests_only():
    s = Scheduler(100, max_inflight=1)
    s.submit(1, 100, 0, deadline_ns=50)        # admitted in time: runs past its deadline
    s.submit(2, 10, 0, deadline_ns=80)
    s.submit(3, 10, 0)
    s.submit(4, 10, 0, deadline_ns=1000)
    slot, ids, exp = s.next(10)
    assert ids == [1] and exp == []
    slot2, ids2, exp2 = s.next(100)            # 2 is due; nothing fits beside 1
    assert (slot2, ids2, exp2) == (-1, [], [2])
    s.complete(slot)
    slot, ids, exp = s.next(2000)
    assert ids == [3] and exp == [4]
    assert s.stats()["expired"] == 2


def test_expiry_cap_defers_admission():
    s = Scheduler(100)
    for i in range(1, 6):
        s.submit(i, 1, 0, deadline_ns=10)
    s.submit(6, 1, 0)
    slot, ids, exp = s.next(20, exp_cap=2)
    assert (slot, ids, exp) == (-1, [], [1, 2])
    slot, ids, exp = s.next(20, exp_cap=2)
    assert (slot, ids, exp) == (-1, [], [3, 4])
    slot, ids, exp = s.next(20, exp_cap=2)
    assert ids == [6] and exp == [5]


def test_drain_returns_queued_in_order():
    s = Scheduler(10, max_inflight=1)
    for i in range(1, 200):
        s.submit(i, 5, 0)
    slot, ids, _ = s.next(0)
    assert ids == [1, 2]
    assert s.drain() == list(range(3, 200))
    assert s.stats()["queued"] == 0
    assert s.complete(slot) == OK
    assert s.next(1) == (-1, [], [])


class Model:
    """The policy in plain Python: FIFO, no overtaking, deadlines, budget, slots."""

    def __init__(self, budget, max_views, max_inflight, max_queued):
        self.budget, self.max_views, self.max_inflight = budget, max_views, max_inflight
        self.max_queued = max_queued
        self.q, self.live, self.slots = [], set(), {}

    def submit(self, i, b, now, dl):
        if b <= 0 or i in self.live:
            return INVALID
        if b > self.budget:
            return OOM
        if len(self.q) >= self.max_queued:
            return BUSY
        self.q.append((i, b, dl))
        self.live.add(i)
        return OK

    def next(self, now, exp_cap):
        exp, keep, more = [], [], False
        for (i, b, dl) in self.q:
            if dl > 0 and now > dl and not more:
                if len(exp) >= exp_cap:
                    more = True
                    keep.append((i, b, dl))
                    continue
                exp.append(i)
                self.live.discard(i)
            else:
                keep.append((i, b, dl))
        self.q = keep
        if more or not self.q:
            return -1, [], exp
        free = [s for s in range(self.max_inflight) if s not in self.slots]
        if not free:
            return -1, [], exp
        reserved = sum(b for b, _ in self.slots.values())
        ids, tot = [], 0
        while self.q and len(ids) < self.max_views and reserved + tot + self.q[0][1] <= self.budget:
            i, b, _ = self.q.pop(0)
            ids.append(i)
            tot += b
        if not ids:
            return -1, [], exp
        self.slots[free[0]] = (tot, ids)
        return free[0], ids, exp

    def complete(self, slot):
        if slot not in self.slots:
            return INVALID
        for i in self.slots.pop(slot)[1]:
            self.live.discard(i)
        return OK


@pytest.mark.parametrize("seed", range(6))
def test_randomized_against_model(seed):
    rng = random.Random(seed)
    cfg = dict(budget_bytes=rng.choice([50, 200, 1000]), max_views_per_batch=rng.choice([1, 3, 8]),
               max_inflight=rng.choice([1, 2, 4]), max_queued=rng.choice([5, 40]))
    s = Scheduler(**cfg)
    m = Model(cfg["budget_bytes"], cfg["max_views_per_batch"], cfg["max_inflight"],
              cfg["max_queued"])
    now, nid = 0, 1
    running = []
    for _ in range(2000):
        now += rng.randint(0, 5)
        op = rng.random()
        if op < 0.45:
            i = nid if rng.random() < 0.95 else rng.randint(1, nid)
            nid += 1
            b = rng.choice([0, 1, 5, 20, 60, cfg["budget_bytes"], cfg["budget_bytes"] + 1])
            dl = rng.choice([0, 0, now + rng.randint(0, 30)])
            assert s.submit(i, b, now, dl) == m.submit(i, b, now, dl)
        elif op < 0.8:
            cap = rng.choice([1, 2, 256])
            got = s.next(now, exp_cap=cap)
            want = m.next(now, cap)
            assert got == want
            if got[0] >= 0:
                running.append(got[0])
        elif running:
            slot = running.pop(rng.randrange(len(running)))
            assert s.complete(slot) == m.complete(slot) == OK
        st = s.stats()
        assert 0 <= st["reserved_bytes"] <= cfg["budget_bytes"]
        assert st["reserved_bytes"] == sum(b for b, _ in m.slots.values())
        assert st["queued"] == len(m.q) and st["inflight_batches"] == len(m.slots)


def test_concurrent_submitters_and_one_consumer():
    """Host threads submit while another admits and completes: every id runs once."""
    s = Scheduler(64, max_views_per_batch=8, max_inflight=3, max_queued=100000)
    n_threads, per = 4, 500
    admitted, stop = [], threading.Event()

    def producer(t):
        for k in range(per):
            assert s.submit(t * per + k + 1, 1 + (k % 7), 0) == OK

    def consumer():
        busy = []
        while not stop.is_set() or s.stats()["queued"] or busy:
            slot, ids, _ = s.next(0)
            if slot >= 0:
                admitted.extend(ids)
                busy.append(slot)
            elif busy:
                assert s.complete(busy.pop(0)) == OK

    ths = [threading.Thread(target=producer, args=(t,)) for t in range(n_threads)]
    c = threading.Thread(target=consumer)
    c.start()
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    stop.set()
    c.join(timeout=60)
    assert not c.is_alive()
    assert sorted(admitted) == list(range(1, n_threads * per + 1))
    # within one producer the admission order is its submission order (FIFO)
    for t in range(n_threads):
        mine = [i for i in admitted if t * per < i <= (t + 1) * per]
        assert mine == sorted(mine)
    st = s.stats()
    assert st["reserved_bytes"] == 0 and st["admitted"] == n_threads * per


def test_struct_sizes():
    import ctypes
    assert ctypes.sizeof(N.occ_sched_stats) == 9 * 8
