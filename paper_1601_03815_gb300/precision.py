"""Reduced-precision storage study: the same seeded run with f stored in FP32,
FP16 and BF16 (arithmetic in FP32, reductions in FP64), errors of E(t),
eps(t) and E(k) stated against the FP32 run, and the step time of each
storage (CUDA events, 20 steps from the seeded field).

Default case: the 256^3 timing field (k0 = 8, Ma = 0.15, Re_lambda = 70),
1000 steps of each scheme, E and eps every 10 steps, E(k) every 200 steps; a
run that goes non-finite is reported with the step of the first non-finite
check (the MRT-LBE run of this field does, in every precision).

    python -m paper_1601_03815_gb300.precision [--N 256 --steps 1000]
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import BF16, DUGKS, F16, F32, KIN_ENONFINITE, LBE_MRT, KinError, Sim

STORAGES = {"f32": F32, "f16": F16, "bf16": BF16}


BYTES_PER_CELL = {F32: 152, F16: 76, BF16: 76}  # 19 loads + 19 stores of the storage type


def time_steps(sim, stream, steps=20, warmup=3):
    """Mean device time of one step (CUDA events on the simulation's stream)."""
    import torch

    sim.step(warmup)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    sim.step(steps)
    b.record(stream)
    b.synchronize()
    return a.elapsed_time(b) / 1000.0 / steps


def run_history(N, scheme, storage, seed=1300, k0=8.0, Ma=0.15, re_lambda=70.0, steps=1000,
                every=10, spectrum_every=200, timing_steps=20):
    """E, eps every `every` steps and E(k) every `spectrum_every` steps, after
    timing `timing_steps` steps from the same field."""
    import torch

    dt = 1.0 if scheme == LBE_MRT else 0.5
    stream = torch.cuda.Stream()
    sim = Sim(N, scheme, 0.01, Ma, dt, storage, stream=stream)
    sim.init_field(seed, k0, re_lambda)
    t = time_steps(sim, stream, timing_steps)
    sim.init_field(seed, k0, re_lambda)
    hist, spec, bad = {}, {}, None
    n = 0
    while n <= steps:
        try:
            if n % spectrum_every == 0:
                E, eps, Ek = sim.stats(spectrum=True)
                spec[n] = Ek
            else:
                E, eps = sim.stats()
        except KinError as exc:
            if exc.code != KIN_ENONFINITE:
                raise
            bad = n
            break
        hist[n] = (E, eps)
        if n < steps:
            sim.step(every)
        n += every
    nu = sim.nu
    sim.close()
    return {"hist": hist, "spec": spec, "nonfinite_at": bad, "nu": nu, "step_s": t,
            "mlups": N ** 3 / t / 1e6, "gbs": BYTES_PER_CELL[storage] * N ** 3 / t / 1e9}


def errors(run, ref, shell_floor=1e-6, upto=None):
    """Max relative errors of E, eps over the checks both runs have (up to step
    `upto`), and of the spectrum shells holding more than shell_floor of the
    peak shell."""
    common = sorted(n for n in set(run["hist"]) & set(ref["hist"]) if upto is None or n <= upto)
    eE = max((abs(run["hist"][n][0] / ref["hist"][n][0] - 1) for n in common), default=None)
    ee = max((abs(run["hist"][n][1] / ref["hist"][n][1] - 1) for n in common), default=None)
    ek = None
    for n in sorted(n for n in set(run["spec"]) & set(ref["spec"]) if upto is None or n <= upto):
        a, b = run["spec"][n], ref["spec"][n]
        m = min(len(a), len(b))
        a, b = a[:m], b[:m]
        sig = b > shell_floor * b.max()
        v = float(np.max(np.abs(a[sig] / b[sig] - 1)))
        ek = v if ek is None else max(ek, v)
    return {"E": eE, "eps": ee, "Ek": ek, "checks": len(common)}


def study(N=256, steps=1000, seed=1300):
    out = {}
    for sname, scheme in (("lbe", LBE_MRT), ("dugks", DUGKS)):
        runs = {k: run_history(N, scheme, st, seed=seed, steps=steps) for k, st in STORAGES.items()}
        ref = runs["f32"]
        res = {"nonfinite_at": {k: r["nonfinite_at"] for k, r in runs.items()},
               "ms_per_step": {k: 1000 * r["step_s"] for k, r in runs.items()},
               "mlups": {k: r["mlups"] for k, r in runs.items()},
               "algorithmic_gbs": {k: r["gbs"] for k, r in runs.items()}}
        bad = [r["nonfinite_at"] for r in runs.values() if r["nonfinite_at"] is not None]
        # a run that blows up is compared only while all runs are smooth: up to
        # 20 steps before the earliest non-finite check
        upto = min(bad) - 20 if bad else None
        res["compared_through_step"] = upto if upto is not None else steps
        for k in ("f16", "bf16"):
            res["%s_vs_f32" % k] = errors(runs[k], ref, upto=upto)
        out[sname] = res
    return {"N": N, "steps": steps, "field": "k0=8, Ma=0.15, Re_lambda=70, seed %d" % seed,
            "schemes": out}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=256)
    ap.add_argument("--steps", type=int, default=1000)
    a = ap.parse_args()
    print(json.dumps(study(a.N, a.steps)))


if __name__ == "__main__":
    main()
