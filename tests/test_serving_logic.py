"""Host logic of the serving loop (admission by footprint, arrival order,
continuous batching, latency accounting) against a fake backend on a
virtual clock; no GPU."""
import numpy as np
import pytest

from paper_1601_03815_gb300.serving import Request, Server, poisson_requests


class VClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)


class FakeBackend:
    """Each active simulation costs N^3 cell updates per step at `rate`
    updates per second of virtual time; the 'state' counts steps taken."""

    def __init__(self, clock, rate=1e9):
        self.clock, self.rate = clock, rate
        self.live = {}
        self.peak_bytes = 0
        self.advances = []

    def footprint(self, req):
        return req.N ** 3 * 200

    def create(self, req):
        h = {"req": req, "steps": 0}
        self.live[id(h)] = h
        self.peak_bytes = max(self.peak_bytes, sum(self.footprint(x["req"]) for x in self.live.values()))
        return h

    def advance(self, handles, n):
        self.advances.append((len(handles), n))
        self.clock.t += sum(h["req"].N ** 3 for h in handles) * n / self.rate
        for h in handles:
            h["steps"] += n

    def finish(self, h, want_f):
        return float(h["steps"]), 0.0, None

    def release(self, h):
        del self.live[id(h)]


def _reqs(n, seed=3):
    rng = np.random.default_rng(seed)
    return [Request(rid=k, N=int(rng.choice([16, 32, 48])), scheme=k % 2, re_lambda=25.0,
                    steps=int(rng.integers(50, 400)), seed=k, arrival=float(k) * 0.01)
            for k in range(n)]


def test_every_request_completes_with_its_own_step_count():
    clk = VClock()
    be = FakeBackend(clk)
    reqs = _reqs(40)
    res, rep = Server(be, hbm_budget=10 ** 9, max_active=8, chunk=25, clock=clk, sleep=clk.sleep).run(reqs)
    assert rep["completed"] == 40 and rep["unfinished"] == 0
    by = {r.rid: r for r in res}
    for q in reqs:
        assert by[q.rid].E == q.steps
        assert by[q.rid].latency > 0 and by[q.rid].admitted >= q.arrival - 1e-12
    assert not be.live


def test_admission_respects_budget_and_slots():
    clk = VClock()
    be = FakeBackend(clk)
    reqs = _reqs(60, seed=4)
    budget = 3 * 48 ** 3 * 200
    res, rep = Server(be, hbm_budget=budget, max_active=5, chunk=10, clock=clk, sleep=clk.sleep).run(reqs)
    assert be.peak_bytes <= budget
    assert max(k for k, _ in be.advances) <= 5
    assert rep["completed"] == 60


def test_admission_keeps_arrival_order():
    clk = VClock()
    be = FakeBackend(clk)
    reqs = _reqs(30, seed=5)
    res, _ = Server(be, hbm_budget=2 * 48 ** 3 * 200, max_active=3, chunk=20, clock=clk,
                    sleep=clk.sleep).run(reqs)
    adm = [r.admitted for r in sorted(res, key=lambda r: r.rid)]
    assert all(b >= a for a, b in zip(adm, adm[1:]))


def test_batching_overlaps_work_of_concurrent_requests():
    clk = VClock()
    be = FakeBackend(clk)
    reqs = [Request(rid=k, N=16, scheme=0, re_lambda=25.0, steps=100, seed=k, arrival=0.0) for k in range(6)]
    _, rep = Server(be, hbm_budget=10 ** 9, max_active=6, chunk=50, clock=clk, sleep=clk.sleep).run(reqs)
    assert be.advances == [(6, 50), (6, 50)]
    assert rep["ticks"] == 2


def test_oversized_request_is_rejected():
    clk = VClock()
    be = FakeBackend(clk)
    r = Request(rid=0, N=64, scheme=0, re_lambda=25.0, steps=10, seed=0, arrival=0.0)
    with pytest.raises(ValueError):
        Server(be, hbm_budget=100, clock=clk, sleep=clk.sleep).run([r])


def test_poisson_requests_are_seeded_and_in_range():
    a = poisson_requests(4.0, 100.0, seed=7)
    b = poisson_requests(4.0, 100.0, seed=7)
    assert [(r.N, r.steps, r.arrival) for r in a] == [(r.N, r.steps, r.arrival) for r in b]
    assert 300 < len(a) < 500
    assert all(r.N in (32, 48, 64, 96, 128) and 500 <= r.steps <= 5000 and 20 <= r.re_lambda <= 50 for r in a)
    assert len({r.seed for r in a}) == len(a)
    gaps = np.diff([0.0] + [r.arrival for r in a])
    assert abs(gaps.mean() - 0.25) < 0.05
