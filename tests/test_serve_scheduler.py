"""Host logic of the solve server, on CPU: admission by footprint and free slots,
arrival order, delivery, per-request failures, and the live submit/future interface.
Solvers are replaced by fakes that count ticks, so no device or library is involved."""
import concurrent.futures
import threading

import numpy as np
import pytest

from paper_1801_02417_gb300 import binding as B
from paper_1801_02417_gb300 import serve


class FakeProblem:
    def __init__(self, fp, ticks, bad=False):
        self.fp, self.ticks, self.bad = fp, ticks, bad

    def footprint(self):
        return self.fp


class Ledger:
    def __init__(self):
        self.lock = threading.Lock()
        self.in_use = self.peak_use = self.live = self.peak_live = 0
        self.order = []

    def open(self, prob):
        with self.lock:
            self.in_use += prob.fp
            self.live += 1
            self.peak_use = max(self.peak_use, self.in_use)
            self.peak_live = max(self.peak_live, self.live)

    def close(self, prob):
        with self.lock:
            self.in_use -= prob.fp
            self.live -= 1


class FakeSolver:
    def __init__(self, prob, ledger):
        self.prob, self.ledger = prob, ledger
        ledger.open(prob)

    def get_stokes(self):
        return np.full((4, 2, 2), float(self.prob.fp), np.float32)

    def close(self):
        self.ledger.close(self.prob)


class FakeActive:
    def __init__(self, rid, prob, solver, arrival, admitted, policy):
        self.rid, self.prob, self.s = rid, prob, solver
        self.arrival, self.admitted = arrival, admitted
        self.used = 0

    def launch(self):
        self.used += 1
        if self.prob.bad == "launch":
            raise B.PolsaraError(B.PS_ENONFINITE, "fake non-finite state")
        return 1

    def advance(self):
        return self.used >= self.prob.ticks


class FakeServer(serve.Server):
    def __init__(self, ledger, **kw):
        super().__init__(**kw)
        self.ledger = ledger

    def _prepare(self, prob):
        if prob.bad == "prepare":
            raise B.PolsaraError(B.PS_EINVAL, "fake rejected measurements")
        with self.ledger.lock:
            self.ledger.order.append(prob)
        return FakeSolver(prob, self.ledger)


@pytest.fixture(autouse=True)
def _fake_active(monkeypatch):
    monkeypatch.setattr(serve, "_Active", FakeActive)


def test_run_respects_budget_slots_and_arrival_order():
    led = Ledger()
    probs = [FakeProblem(fp=10 + (i % 3) * 5, ticks=1 + i % 4) for i in range(12)]
    srv = FakeServer(led, hbm_budget=40, max_active=3, prep_workers=1)
    res = srv.run([(0.001 * i, p) for i, p in enumerate(probs)])
    assert sorted(r.rid for r in res) == list(range(12))
    assert led.peak_use <= 40 and led.peak_live <= 3 and led.in_use == 0
    assert led.order == probs                         # one preparation worker: admission order
    for r in res:
        assert r.iterations == probs[r.rid].ticks
        assert r.arrival <= r.admitted <= r.finished
        assert r.S[0, 0, 0] == probs[r.rid].fp


def test_oversized_request_runs_alone():
    led = Ledger()
    probs = [FakeProblem(10, 2), FakeProblem(100, 2), FakeProblem(10, 2)]
    res = FakeServer(led, hbm_budget=50, max_active=8).run([(0.0, p) for p in probs])
    assert len(res) == 3 and led.peak_use <= 100 and led.in_use == 0


def test_run_raises_a_failed_request():
    led = Ledger()
    probs = [FakeProblem(10, 2), FakeProblem(10, 2, bad="prepare")]
    with pytest.raises(B.PolsaraError):
        FakeServer(led, hbm_budget=100).run([(0.0, p) for p in probs])


def test_live_submit_resolves_futures_and_isolates_failures():
    led = Ledger()
    probs = [FakeProblem(5 + i, 1 + i % 5) for i in range(20)]
    probs[4] = FakeProblem(7, 3, bad="prepare")
    probs[9] = FakeProblem(7, 3, bad="launch")
    with FakeServer(led, hbm_budget=30, max_active=4, prep_workers=2) as srv:
        with concurrent.futures.ThreadPoolExecutor(5) as ex:
            futs = list(ex.map(srv.submit, probs))
        for i, f in enumerate(futs):
            if probs[i].bad:
                with pytest.raises(B.PolsaraError) as e:
                    f.result(timeout=30)
                assert e.value.status == (B.PS_EINVAL if probs[i].bad == "prepare" else B.PS_ENONFINITE)
            else:
                r = f.result(timeout=30)
                assert r.iterations == probs[i].ticks and r.S[0, 0, 0] == probs[i].fp
    assert led.peak_use <= 30 and led.peak_live <= 4 and led.in_use == 0
    with pytest.raises(RuntimeError):
        srv.submit(probs[0])


def test_submit_requires_start_and_stop_is_idempotent():
    srv = FakeServer(Ledger(), hbm_budget=10)
    with pytest.raises(RuntimeError):
        srv.submit(FakeProblem(1, 1))
    srv.stop()
    srv.start()
    f = srv.submit(FakeProblem(1, 2))
    srv.stop()
    assert f.result(timeout=5).iterations == 2
    srv.stop()
