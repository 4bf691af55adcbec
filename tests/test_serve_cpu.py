"""Admission control of the serving loop on CPU: plans held under an HBM
budget, idle plans evicted least-recently-used first, busy plans never
evicted, and no admission while nothing can be freed.  The plan object is a
stand-in recording its size and closure; no GPU and no estimator work."""
import collections
import time

import numpy as np
import pytest

pytest.importorskip("torch")
from paper_1705_06284_gb300 import serve


class FakePlan:
    closed = []
    counts_seen = []
    gate = None  # a threading.Event the constructor waits on (slow builds)

    def __init__(self, N, L, edges, precision="bf16x3", stream=None, counts=None):
        if FakePlan.gate is not None and N == 16:
            FakePlan.gate.wait(5.0)
        self.N, self.device_bytes = N, 1000 * N
        self.stream = stream
        self.triplets = np.zeros((0, 3), dtype=np.int32)
        self.N_tri = np.zeros(0, dtype=np.int64)
        FakePlan.counts_seen.append(counts)

    def export_counts(self):
        return b"counts-%d" % self.N

    def set_stream(self, s):
        self.stream = s

    def close(self):
        FakePlan.closed.append(self.N)


def _server(budget, monkeypatch, pool=None):
    monkeypatch.setattr(serve, "Plan", FakePlan)
    monkeypatch.setattr(serve, "plan_bytes_estimate", lambda N, nbins, slab_budget=0: 1000 * N)
    srv = serve.EstimatorServer.__new__(serve.EstimatorServer)
    srv.budget, srv.held, srv.plan_creations, srv.plans_from_cache = budget, 0, 0, 0
    srv.plans = collections.defaultdict(list)
    srv.slots, srv._cancelled = [], set()
    srv.counts_cache, srv.count_cache_dir, srv.slab_bytes = {}, None, 1 << 30
    srv.FRESH_S = 0.0  # new plans evictable at once (the pin has its own test)
    srv._building, srv._pool, srv._build_stream, srv._failed = {}, pool, None, {}
    FakePlan.closed, FakePlan.counts_seen, FakePlan.gate = [], [], None
    return srv


def _req(rid, N, nb=4):
    return serve.Request(rid, np.zeros((N, N, N), dtype=np.float32), 100.0, tuple(range(nb + 1)))


def test_admission_eviction_and_reuse(monkeypatch):
    f8 = 2 * 8 ** 3 * 4  # two staging copies of an 8^3 field
    srv = _server(3 * (8000 + f8), monkeypatch)
    e1 = srv._plan_for(_req(1, 8), "s1")
    e1["last"] = 1.0
    e2 = srv._plan_for(_req(2, 8, nb=5), "s2")
    e2["last"] = 2.0
    e3 = srv._plan_for(_req(3, 8, nb=6), "s3")
    e3["last"] = 3.0
    assert srv.plan_creations == 3 and srv.held == 3 * (8000 + f8)
    # the same key reuses its idle plan on the new stream
    again = srv._plan_for(_req(4, 8), "s4")
    assert again is e1 and e1["plan"].stream == "s4" and srv.plan_creations == 3
    # a fourth key: the least recently used idle plan (e1) is evicted
    e4 = srv._plan_for(_req(5, 8, nb=7), "s5")
    assert e4 is not None and FakePlan.closed == [8] and srv.held == 3 * (8000 + f8)
    assert srv.plans[(8, 100.0, tuple(float(v) for v in range(5)), "bf16x3")] == []


def test_busy_plans_are_never_evicted(monkeypatch):
    f8 = 2 * 8 ** 3 * 4
    srv = _server(2 * (8000 + f8), monkeypatch)
    a = srv._plan_for(_req(1, 8), "s1")
    b = srv._plan_for(_req(2, 8, nb=5), "s2")
    a["busy"] = b["busy"] = True
    assert srv._plan_for(_req(3, 8, nb=6), "s3") is None  # nothing idle to free
    assert FakePlan.closed == [] and srv.held == 2 * (8000 + f8)
    b["busy"] = False
    assert srv._plan_for(_req(4, 8, nb=6), "s4") is not None and FakePlan.closed == [8]


def test_request_larger_than_the_budget_is_refused_not_stuck(monkeypatch):
    f8 = 2 * 8 ** 3 * 4
    srv = _server(8000 + f8, monkeypatch)
    # needs 16000 + its field copies: more than the whole budget
    assert srv._plan_for(_req(1, 16), "s1") is srv.NEVER
    # fits the budget but not beside a busy plan: wait, do not refuse
    a = srv._plan_for(_req(2, 8), "s2")
    a["busy"] = True
    assert srv._plan_for(_req(3, 8, nb=5), "s3") is None
    a["busy"] = False
    assert srv._plan_for(_req(4, 8, nb=5), "s4") is not None


class _FakeSlot:
    def __init__(self):
        self.stream, self.busy = "s", None


def test_run_refuses_oversize_and_cancelled_requests(monkeypatch):
    f8 = 2 * 8 ** 3 * 4
    srv = _server(8000 + f8, monkeypatch)
    srv.slots = [_FakeSlot()]
    served = []

    def fake_submit(slot, req, entry, t0):  # completes at once, no GPU
        served.append(req.rid)

    monkeypatch.setattr(srv, "_submit", fake_submit)
    srv.cancel(3)
    res = srv.run([_req(1, 16), _req(2, 8), _req(3, 8, nb=5)], realtime=False)
    errs = {r.rid: r.error for r in res}
    assert errs[1] == "does not fit the HBM budget"
    assert errs[3] == "cancelled"
    assert served == [2]


class _Done:
    def query(self):
        return True


def test_plan_builds_do_not_hold_up_admission(monkeypatch):
    """A request whose plan is being built (slowly, on the builder thread)
    does not stop the loop: a later request with a ready plan is admitted and
    completes first; the first is admitted once its plan exists."""
    import concurrent.futures
    import threading
    import torch
    pool = concurrent.futures.ThreadPoolExecutor(max_workers=1)
    srv = _server(10 ** 9, monkeypatch, pool=pool)
    srv.slots = [_FakeSlot(), _FakeSlot()]
    order = []

    def fake_submit(slot, req, entry, t0):
        order.append(req.rid)
        entry["busy"] = True
        slot.busy = (req, entry, _Done(), (None, None, torch.zeros(0), torch.zeros(0), None), 0.0)

    monkeypatch.setattr(srv, "_submit", fake_submit)
    srv._plan_for(_req(0, 8), "s")  # the 8^3 plan is built and resident before the run
    deadline = time.time() + 5
    while srv._building and time.time() < deadline:
        srv._poll_builds()
    FakePlan.gate = threading.Event()
    timer = threading.Timer(0.3, FakePlan.gate.set)
    timer.start()
    res = srv.run([_req(1, 16), _req(2, 8)], realtime=False)
    timer.join()
    pool.shutdown()
    assert order == [2, 1]  # 2 went ahead while 1's plan was being built
    assert sorted(r.rid for r in res) == [1, 2] and all(r.error is None for r in res)
    assert srv.plan_creations == 2


def test_rebuilt_plans_take_their_counts_from_the_cache(monkeypatch):
    f8 = 2 * 8 ** 3 * 4
    srv = _server(8000 + f8, monkeypatch)
    e1 = srv._plan_for(_req(1, 8), "s1")          # built from scratch, counts kept
    assert FakePlan.counts_seen == [None] and srv.plans_from_cache == 0
    e2 = srv._plan_for(_req(2, 8, nb=5), "s2")    # another key evicts the first
    assert e2 is not None and FakePlan.closed == [8]
    e3 = srv._plan_for(_req(3, 8), "s3")          # the first key again: from its counts
    assert FakePlan.counts_seen[-1] == b"counts-8" and srv.plans_from_cache == 1


def test_deadline_refuses_requests_not_yet_admitted(monkeypatch):
    f8 = 2 * 8 ** 3 * 4
    srv = _server(4 * (8000 + f8), monkeypatch)
    srv.slots = [_FakeSlot()]
    served = []

    def fake_submit(slot, req, entry, t0):
        served.append(req.rid)

    monkeypatch.setattr(srv, "_submit", fake_submit)
    reqs = [_req(1, 8), _req(2, 8, nb=5)]
    reqs[1].arrival = 0.5  # arrives after the deadline
    res = srv.run(reqs, realtime=True, deadline_s=0.05)
    errs = {r.rid: r.error for r in res}
    assert served == [1] and errs == {2: "deadline"}  # the stand-in submit leaves no result for 1


def test_new_plans_are_kept_for_their_request(monkeypatch):
    """A plan built for a waiting request is not evicted for another request's
    plan before its first use (no build-evict cycles under a tight budget)."""
    f8 = 2 * 8 ** 3 * 4
    srv = _server(8000 + f8, monkeypatch)
    srv.FRESH_S = 60.0
    a = srv._plan_for(_req(1, 8), "s1")
    assert a is not None
    # a second key needs the same room: it must wait, the fresh plan stays
    assert srv._plan_for(_req(2, 8, nb=5), "s2") is None  # waits, is not refused
    assert FakePlan.closed == []
    a["fresh_until"] = 0.0  # used once: evictable again
    b = srv._plan_for(_req(2, 8, nb=5), "s2")
    assert b is not None and FakePlan.closed == [8]
