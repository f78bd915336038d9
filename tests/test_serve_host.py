"""Serving loop admission and failure handling on the host (fake executor,
no GPU): the byte budget is never exceeded, oversize requests are rejected,
a failing request does not stop the others, small SV requests are batched."""
import threading
import time

import numpy as np
import pytest

from paper_2401_06861_gb300 import _lib as L
from paper_2401_06861_gb300 import inputs
from paper_2401_06861_gb300.serve import Server, state_bytes, summarize


class FakeStream:
    cuda_stream = 0


class FakeExecutor:
    def __init__(self, ledger_probe=None, fail_ids=(), delay=0.002):
        self.fail_ids = set(fail_ids)
        self.delay = delay
        self.max_used = 0
        self.batches = []
        self.server = None
        self.lock = threading.Lock()

    def new_stream(self):
        return FakeStream()

    def _result(self, r):
        return dict(z=np.full(r["n"], float(r["id"])), energy=-float(r["id"]))

    def run_single(self, req, stream):
        with self.lock:
            self.max_used = max(self.max_used, self.server.ledger.used)
            assert self.server.ledger.used <= self.server.ledger.budget
        time.sleep(self.delay)
        if req["id"] in self.fail_ids:
            raise RuntimeError("injected failure")
        return self._result(req)

    def run_batch(self, reqs, stream):
        self.batches.append([r["id"] for r in reqs])
        time.sleep(self.delay)
        return [self._result(r) for r in reqs]


def make(ex, **kw):
    srv = Server(ex, **kw)
    ex.server = srv
    return srv


def test_budget_is_never_exceeded_and_all_requests_complete():
    reqs = inputs.serve_requests(rate=2000, duration=0.1, seed=1, sv_n=(8, 20), dm_n=(6, 9))
    budget = 3 * state_bytes(dict(kind="sv", n=20), L.F32)
    ex = FakeExecutor()
    srv = make(ex, budget_bytes=budget, slots=6, batch_max_n=12)
    res = srv.serve(reqs, realtime=True)
    assert len(res) == len(reqs)
    assert all(r["error"] is None for r in res.values())
    assert srv.ledger.peak <= budget and srv.ledger.used == 0
    # small SV requests went through batches, the others through streams
    for r in reqs:
        want = "batch" if (r["kind"] == "sv" and r["n"] <= 12) else "stream"
        assert res[r["id"]]["path"] == want
        assert res[r["id"]]["energy"] == -r["id"]
    s = summarize(res, srv.wall)
    assert s["completed"] == len(reqs) and s["p99_ms"] >= s["p50_ms"] > 0


def test_oversize_request_rejected_and_failure_isolated():
    reqs = inputs.serve_requests(rate=1000, duration=0.05, seed=2, sv_n=(13, 16), dm_n=(6, 7))
    big = dict(reqs[0], id=len(reqs), n=30, kind="sv", arrival=0.001)
    reqs = reqs + [big]
    ex = FakeExecutor(fail_ids={reqs[1]["id"]})
    srv = make(ex, budget_bytes=state_bytes(dict(kind="sv", n=20), L.F32), slots=3, batch_max_n=0)
    res = srv.serve(reqs)
    assert res[big["id"]]["error"].startswith("EBUDGET")
    assert "injected failure" in res[reqs[1]["id"]]["error"]
    others = [r for r in reqs if r["id"] not in (big["id"], reqs[1]["id"])]
    assert all(res[r["id"]]["error"] is None for r in others)


def test_delayed_and_dropped_arrivals():
    reqs = inputs.serve_requests(rate=500, duration=0.1, seed=3, sv_n=(8, 14), dm_n=(6, 7))
    rng = np.random.default_rng(0)
    kept = [dict(r, arrival=r["arrival"] + rng.uniform(0, 0.02)) for r in reqs if rng.random() > 0.2]
    ex = FakeExecutor()
    srv = make(ex, slots=2, batch_max_n=10)
    res = srv.serve(kept)
    assert sorted(res) == sorted(r["id"] for r in kept)
    assert all(r["error"] is None for r in res.values())
