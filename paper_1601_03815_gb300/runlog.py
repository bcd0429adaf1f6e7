"""JSON-lines run log of a simulation: the quantities the paper records over a
decay run (Sec. III: E, eps, E(k); Eqs. 26, 27) at their cadences.

    run_logged(sim, steps, "run.jsonl", stats_every=10, spectrum_every=200)

writes one object per line:
    {"kind": "run", ...}                      the simulation's parameters
    {"kind": "stats", "step", "t", "E", "eps"[, "Ek"]}
                                              every stats_every steps (and at
                                              step 0); E(k) every spectrum_every
    {"kind": "summary", "steps", "seconds", "mlups", "gbs"}
                                              wall time of the whole run, cell
                                              updates per second and the
                                              algorithmic bytes moved per second
The statistics of a logged step come from kin_step_stats, so the fused DUGKS
step leaves the velocity they need and no separate pass is paid.
"""
from __future__ import annotations

import json
import time

BYTES_PER_CELL = {0: 152, 1: 76, 2: 76, 3: 304}  # 19 loads + 19 stores of the storage type
SCHEMES = {0: "lbe", 1: "dugks"}
STORAGES = {0: "f32", 1: "f16", 2: "bf16", 3: "f64"}


def run_logged(sim, steps: int, out, stats_every: int = 10, spectrum_every: int = 200) -> dict:
    """Advance `sim` by `steps` steps, logging to `out` (a path or an open text
    file).  Returns the summary record."""
    if stats_every <= 0 or steps < 0:
        raise ValueError("stats_every must be positive and steps non-negative")
    fh = open(out, "w") if isinstance(out, str) else out
    try:
        fh.write(json.dumps({"kind": "run", "N": sim.N, "scheme": SCHEMES[sim.scheme],
                             "storage": STORAGES[sim.storage], "nu": sim.nu, "dt": sim.dt,
                             "stats_every": stats_every, "spectrum_every": spectrum_every}) + "\n")

        def record(step, stats):
            rec = {"kind": "stats", "step": step, "t": sim.time, "E": stats[0], "eps": stats[1]}
            if len(stats) > 2:
                rec["Ek"] = [float(v) for v in stats[2]]
            fh.write(json.dumps(rec) + "\n")

        spec0 = spectrum_every > 0
        record(sim.steps_taken, sim.stats(spectrum=spec0))
        t0 = time.perf_counter()
        done = 0
        while done < steps:
            n = min(stats_every - done % stats_every, steps - done)
            done += n
            spec = spectrum_every > 0 and done % spectrum_every == 0
            if done % stats_every == 0 or done == steps:
                stats = sim.step_stats(n, spectrum=spec)
                record(sim.steps_taken, stats)
            else:
                sim.step(n)
        sim.sync()
        dt = time.perf_counter() - t0
        cells = sim.N ** 3 * steps
        summary = {"kind": "summary", "steps": steps, "seconds": dt,
                   "mlups": cells / dt / 1e6 if dt > 0 else None,
                   "gbs": cells * BYTES_PER_CELL[sim.storage] / dt / 1e9 if dt > 0 else None}
        fh.write(json.dumps(summary) + "\n")
        return summary
    finally:
        if isinstance(out, str):
            fh.close()
