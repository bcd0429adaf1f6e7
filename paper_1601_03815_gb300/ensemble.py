"""Batched ensembles: independent DHIT realisations of uneven N advanced by one
CUDA graph launch per call (a persistent kernel for the DUGKS members, beside
it one batched launch per step for the LBE members), with an autotuner for
the work decomposition (DUGKS plane-tile height and z chunk, threads per block
of the batched LBE launches).

The reference ensemble has 24 members, 8 x 32^3, 8 x 64^3, 6 x 96^3 and
2 x 128^3, each with its own seed, a seeded coin for the scheme, Ma = 0.1 and
Re_lambda drawn uniformly from [20, 40].

    python -m paper_1601_03815_gb300.ensemble [--steps 500]

prints one JSON line: the batched aggregate MLUPS against the sum of the same
members stepped one by one with kin_step.
"""
from __future__ import annotations

import argparse
import itertools
import json
import os
import time

import numpy as np

from . import DUGKS, F32, LBE_MRT, Ensemble, Sim

REFERENCE_SIZES = ((32, 8), (64, 8), (96, 6), (128, 2))
TUNE_TILE_Y = (4, 6, 8)
TUNE_ZCHUNK = (8, 16, 32, 64, 128)
TUNE_LBE_BLOCK = (64, 128)


def member_specs(sizes=REFERENCE_SIZES, seed: int = 1400, re_range=(20.0, 40.0)):
    """(N, scheme, seed, Re_lambda) of every member, from a seeded generator."""
    rng = np.random.default_rng(seed)
    specs = []
    k = 0
    for N, count in sizes:
        for _ in range(count):
            scheme = LBE_MRT if rng.random() < 0.5 else DUGKS
            specs.append((N, scheme, seed + 1 + k, float(rng.uniform(*re_range))))
            k += 1
    return specs


def make_members(specs, Ma: float = 0.1, k0: float = 4.0, dugks_dt: float = 0.5):
    sims = []
    for N, scheme, seed, re in specs:
        s = Sim(N, scheme, 0.01, Ma, 1.0 if scheme == LBE_MRT else dugks_dt, F32)
        s.init_field(seed, k0, re)
        sims.append(s)
    return sims


def _cache_path():
    base = os.environ.get("KIN_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "kin_ensemble_tuning.json")


def _signature(sims):
    import torch

    dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    sizes = sorted((s.N, s.scheme) for s in sims)
    # "c": tunings of the batched-LBE form (threads per LBE block, 6-row tiles)
    return "c|%s|%s" % (dev, ",".join("%d%s" % (n, "L" if sc == LBE_MRT else "D") for n, sc in sizes))


def autotune(ens: Ensemble, steps: int = 10, use_cache: bool = True, verbose: bool = False):
    """Time every (tile_y, zchunk, lbe_block) candidate on this ensemble and
    leave the fastest set.  The members advance while tuning.  Results are
    cached per device and member mix."""
    sig = _signature(ens.members)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as fh:
                cache = json.load(fh)
        except Exception:
            cache = {}
    if use_cache and sig in cache:
        best = cache[sig]
        ens.set_tuning(*best["tuning"])
        return best
    timings = []
    for ty, zc, ln in itertools.product(TUNE_TILE_Y, TUNE_ZCHUNK, TUNE_LBE_BLOCK):
        ens.set_tuning(ty, zc, ln)
        ens.step(2)  # capture the graph and warm up
        t0 = time.perf_counter()
        ens.step(steps)
        dt = time.perf_counter() - t0
        timings.append((dt, (ty, zc, ln)))
        if verbose:
            print("tile_y=%d zchunk=%d lbe_block=%d: %.3f ms/step" % (ty, zc, ln, 1e3 * dt / steps))
    dt, tuning = min(timings)
    ens.set_tuning(*tuning)
    best = {"tuning": list(tuning), "ms_per_step": 1e3 * dt / steps,
            "candidates": [[list(t), 1e3 * d / steps] for d, t in timings]}
    if use_cache:
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            cache[sig] = best
            with open(path, "w") as fh:
                json.dump(cache, fh)
        except Exception:
            pass
    return best


def measure(steps: int = 500, seed: int = 1400, tune: bool = True, verbose: bool = False):
    """Batched vs one-by-one aggregate throughput of the reference ensemble."""
    import torch

    specs = member_specs(seed=seed)
    cells = sum(N ** 3 for N, _, _, _ in specs)
    sims = make_members(specs)
    ens = Ensemble(sims)
    tuned = autotune(ens, verbose=verbose) if tune else None
    # restart from the seeded fields for the timed run
    for s, (N, scheme, sd, re) in zip(sims, specs):
        s.init_field(sd, 4.0, re)
    ens.step(steps)  # captures the graph for this step count (untimed)
    for s, (N, scheme, sd, re) in zip(sims, specs):
        s.init_field(sd, 4.0, re)
    torch.cuda.synchronize()
    launches0 = ens.info()["launches"]
    t0 = time.perf_counter()
    ens.step(steps)
    t_batched = time.perf_counter() - t0
    graph_launches = ens.info()["launches"] - launches0
    stats = [s.stats() for s in sims]
    # the same members one by one with kin_step (their own launches)
    for s, (N, scheme, sd, re) in zip(sims, specs):
        s.init_field(sd, 4.0, re)
    t_plain = 0.0
    for s in sims:
        s.step(2)
        s.sync()
        t0 = time.perf_counter()
        s.step(steps)
        s.sync()
        t_plain += time.perf_counter() - t0
    info = ens.info()
    ens.close()
    for s in sims:
        s.close()
    return {
        "members": len(specs), "cells_per_step": cells, "steps": steps,
        "batched_mlups": cells * steps / t_batched / 1e6,
        "batched_s": t_batched,
        "one_by_one_mlups": cells * steps / t_plain / 1e6,
        "one_by_one_s": t_plain,
        "graph_launches": graph_launches,
        "kernels": {"persistent_dugks_per_graph": 1 if any(sp[1] == DUGKS for sp in specs) else 0,
                    "batched_lbe_per_step": 1 if any(sp[1] == LBE_MRT for sp in specs) else 0},
        "graph": True, "tuning": tuned["tuning"] if tuned else None,
        "items_per_step": info["items"], "blocks": info["grid"],
        "schemes": {"lbe": sum(1 for sp in specs if sp[1] == LBE_MRT),
                    "dugks": sum(1 for sp in specs if sp[1] == DUGKS)},
        "finite": all(np.isfinite(e) and np.isfinite(p) for e, p in stats),
    }


def just_step(steps: int, tuning, seed: int = 1400):
    """Build the reference ensemble, set `tuning` (tile_y, zchunk, lbe_block)
    and advance it `steps` steps in one call, untimed (for profilers)."""
    import torch

    sims = make_members(member_specs(seed=seed))
    ens = Ensemble(sims)
    ens.set_tuning(*tuning)
    ens.step(steps)
    torch.cuda.synchronize()
    info = ens.info()
    ens.close()
    for s in sims:
        s.close()
    return info


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--seed", type=int, default=1400)
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--verbose", action="store_true")
    ap.add_argument("--just-step", type=int, default=0, metavar="K",
                    help="only advance the reference ensemble K steps in one call (for profilers)")
    ap.add_argument("--tuning", type=int, nargs=3, default=[6, 128, 128], metavar=("TILE_Y", "ZCHUNK", "LBE_BLOCK"))
    a = ap.parse_args()
    if a.just_step > 0:
        print(json.dumps(just_step(a.just_step, a.tuning, a.seed)))
        return
    print(json.dumps(measure(a.steps, a.seed, not a.no_tune, a.verbose)))


if __name__ == "__main__":
    main()
