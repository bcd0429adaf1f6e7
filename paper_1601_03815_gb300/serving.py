"""Serving loop with continuous batching of simulation requests.

A request asks for one DHIT simulation: (N, scheme, Re_lambda, steps, seed).
The server admits queued requests in arrival order while their device
footprint fits the HBM budget and a slot is free, keeps every admitted state
resident, and advances all active simulations together, a chunk of steps per
tick.  A request that arrives while others run joins at the next tick; a
finished one is read out (E, eps and optionally f), freed, and its memory and
slot go to the queue.

Two backends advance a tick.  StreamBackend (the default) enqueues every
active simulation's steps on its own stream with kin_step, so the tuned
single-simulation kernels of all requests run concurrently on the device;
GpuBackend advances them in one persistent ensemble launch
(kin_ensemble_step).  A simulation's arithmetic does not depend on the other
requests or on how its steps are grouped, so with either backend a request's
result is bitwise the same alone and in any mix.  On the reference workload
the stream backend halves the median latency (the ensemble kernel's items run
below the standalone kernels: one 10-warp block per SM for the memory-bound
LBE items).

    python -m paper_1601_03815_gb300.serving --seconds 600 --rate 4 [--backend ensemble]

runs the reference workload (Poisson arrivals at `rate` per second, N uniform
over {32, 48, 64, 96, 128}, LBE or DUGKS 50/50, Re_lambda uniform in [20, 50],
steps uniform in [500, 5000], distinct seeds) and prints p50 / p99
time-to-completion and aggregate MLUPS as one JSON line.
"""
from __future__ import annotations

import argparse
import collections
import dataclasses
import json
import time

import numpy as np

SIZES = (32, 48, 64, 96, 128)


@dataclasses.dataclass
class Request:
    rid: int
    N: int
    scheme: int            # 0 = LBE, 1 = DUGKS
    re_lambda: float
    steps: int
    seed: int
    arrival: float         # seconds from the start of the run
    Ma: float = 0.1
    k0: float = 4.0
    want_f: bool = False


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    done: float
    steps: int
    cells: int
    E: float
    eps: float
    f: object = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def poisson_requests(rate: float, seconds: float, seed: int = 2024, sizes=SIZES,
                     steps=(500, 5000), re_range=(20.0, 50.0)):
    """Seeded Poisson arrivals over [0, seconds)."""
    rng = np.random.default_rng(seed)
    t, out, k = 0.0, [], 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= seconds:
            break
        out.append(Request(rid=k, N=int(rng.choice(sizes)), scheme=int(rng.random() < 0.5),
                           re_lambda=float(rng.uniform(*re_range)),
                           steps=int(rng.integers(steps[0], steps[1] + 1)),
                           seed=seed * 1000 + k, arrival=t))
        k += 1
    return out


class GpuBackend:
    """Simulations in libkin; active ones advance by one ensemble launch."""

    def __init__(self, tuning=None):
        from . import DUGKS, F32, LBE_MRT, footprint_bytes

        self._fp = footprint_bytes
        self._consts = (DUGKS, F32, LBE_MRT)
        self.tuning = tuning
        self._ens = None
        self._ens_key = None

    def footprint(self, req: Request) -> int:
        # state buffers + statistics scratch (u: 3 N^3 doubles, spectrum arrays)
        N = req.N
        return self._fp(N, req.scheme, self._consts[1]) + 3 * N ** 3 * 8 + 3 * N * N * (N // 2 + 1) * 16

    def create(self, req: Request):
        from . import Sim

        DUGKS, F32, LBE_MRT = self._consts
        sim = Sim(req.N, req.scheme, 0.01, req.Ma, 1.0 if req.scheme == LBE_MRT else 0.5, F32)
        sim.init_field(req.seed, req.k0, req.re_lambda)
        return sim

    def advance(self, sims, nsteps: int):
        from . import Ensemble

        key = tuple(id(s) for s in sims)
        if key != self._ens_key:
            if self._ens is not None:
                self._ens.close()
            self._ens = Ensemble(sims)
            if self.tuning:
                self._ens.set_tuning(*self.tuning)
            self._ens_key = key
        self._ens.step(nsteps)

    def finish(self, sim, want_f: bool):
        E, eps = sim.stats()
        f = sim.get_f() if want_f else None
        return E, eps, f

    def release(self, sim):
        if self._ens is not None and any(s is sim for s in self._ens.members):
            self._ens.close()
            self._ens, self._ens_key = None, None
        sim.close()

    def close(self):
        if self._ens is not None:
            self._ens.close()
            self._ens, self._ens_key = None, None


class StreamBackend(GpuBackend):
    """Simulations in libkin, each on its own stream; a tick enqueues n steps
    of every active simulation, then waits for all of them."""

    def advance(self, sims, nsteps: int):
        for s in sims:
            s.step(nsteps)
        for s in sims:
            s.sync()

    def release(self, sim):
        sim.close()

    def close(self):
        pass


BACKENDS = {"streams": StreamBackend, "ensemble": GpuBackend}


class Server:
    def __init__(self, backend, hbm_budget: int, max_active: int = 64, chunk: int = 50,
                 clock=time.perf_counter, sleep=time.sleep):
        self.backend = backend
        self.budget = int(hbm_budget)
        self.max_active = max_active
        self.chunk = chunk
        self.clock = clock
        self.sleep = sleep

    def run(self, requests, duration: float | None = None):
        """Serve `requests` (arrival times relative to the start); returns
        (results, report).  With `duration`, stops admitting and stepping once
        the wall time passes it."""
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        queue = collections.deque()
        active = []  # dicts: req, handle, remaining, admitted, bytes
        results = []
        used = 0
        t0 = self.clock()
        cell_updates = 0
        ticks = 0
        max_active_seen = 0
        while pending or queue or active:
            now = self.clock() - t0
            if duration is not None and now >= duration:
                break
            while pending and pending[0].arrival <= now:
                queue.append(pending.popleft())
            # admission in arrival order (no overtaking), by footprint and slots
            while queue and len(active) < self.max_active:
                req = queue[0]
                need = self.backend.footprint(req)
                if need > self.budget:
                    raise ValueError("request %d needs %d bytes, budget is %d" % (req.rid, need, self.budget))
                if used + need > self.budget:
                    break
                queue.popleft()
                handle = self.backend.create(req)
                used += need
                active.append({"req": req, "handle": handle, "remaining": req.steps,
                               "admitted": self.clock() - t0, "bytes": need})
            max_active_seen = max(max_active_seen, len(active))
            if not active:
                if pending:
                    self.sleep(max(0.0, min(pending[0].arrival - (self.clock() - t0), 0.05)))
                continue
            n = min(self.chunk, min(a["remaining"] for a in active))
            self.backend.advance([a["handle"] for a in active], n)
            ticks += 1
            for a in active:
                a["remaining"] -= n
                cell_updates += a["req"].N ** 3 * n
            still = []
            for a in active:
                if a["remaining"] == 0:
                    req = a["req"]
                    E, eps, f = self.backend.finish(a["handle"], req.want_f)
                    self.backend.release(a["handle"])
                    used -= a["bytes"]
                    results.append(Result(req.rid, req.arrival, a["admitted"], self.clock() - t0,
                                          req.steps, req.N ** 3, E, eps, f))
                else:
                    still.append(a)
            active = still
        wall = self.clock() - t0
        for a in active:
            self.backend.release(a["handle"])
        lat = np.array([r.latency for r in results]) if results else np.zeros(0)
        report = {
            "completed": len(results), "submitted": len(requests),
            "unfinished": len(active) + len(queue) + len(pending),
            "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
            "mean_s": float(lat.mean()) if lat.size else None,
            "aggregate_mlups": cell_updates / wall / 1e6 if wall > 0 else None,
            "completed_mlups": sum(r.cells * r.steps for r in results) / wall / 1e6 if wall > 0 else None,
            "wall_s": wall, "ticks": ticks, "max_active": max_active_seen,
            "chunk": self.chunk, "hbm_budget_bytes": self.budget,
        }
        return results, report


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--seconds", type=float, default=600.0, help="arrival window")
    ap.add_argument("--rate", type=float, default=4.0)
    ap.add_argument("--seed", type=int, default=2024)
    ap.add_argument("--chunk", type=int, default=50)
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--max-active", type=int, default=64)
    ap.add_argument("--backend", choices=sorted(BACKENDS), default="streams")
    a = ap.parse_args()
    import torch

    from . import load

    load()
    torch.cuda.init()
    reqs = poisson_requests(a.rate, a.seconds, a.seed)
    backend = BACKENDS[a.backend]()
    srv = Server(backend, int(a.budget_gb * 2 ** 30), a.max_active, a.chunk)
    results, report = srv.run(reqs, duration=None)
    backend.close()
    report.update({"backend": a.backend, "rate_per_s": a.rate, "arrival_window_s": a.seconds, "seed": a.seed,
                   "finite": all(np.isfinite(r.E) for r in results)})
    print(json.dumps(report))


if __name__ == "__main__":
    main()
