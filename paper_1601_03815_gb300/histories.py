"""Decay histories of the two schemes from one initial field (Sec. IV: the
paper's runs at Re_lambda = 26.06, 52.12 and 104.24 on 128^3).

Both schemes start from the same seeded field (spectrum shape
k^4 exp(-0.14 k^2), u' = 0.032) with nu from Re_lambda.  Time is measured in
lattice units; MRT-LBE advances dt = 1 per step and DUGKS dt = 0.5 (CFL
0.7071), so DUGKS takes two steps per LBE step.  E and eps (grid form) are
recorded every `every` time units, the derived statistics (lambda, Re_lambda,
eta, S, F) every `derived_every`, and the largest relative difference of E
and eps between the schemes is reported.

    python -m paper_1601_03815_gb300.histories [--N 128 --time 2000 --re 52.12,104.24]
"""
from __future__ import annotations

import argparse
import json
import math

from . import DUGKS, F32, LBE_MRT, Sim

RS = math.sqrt(1.0 / 3.0)
K0 = math.sqrt(2.0 / 0.14)
U_PRIME = 0.032


def history(N: int, re_lambda: float, T: int, every: int = 20, derived_every: int = 500, seed: int = 1700,
            k0: float = K0):
    out = {}
    for name, scheme, dt in (("lbe", LBE_MRT, 1.0), ("dugks", DUGKS, 0.5)):
        per = int(round(1.0 / dt))  # steps per lattice time unit
        sim = Sim(N, scheme, 0.01, U_PRIME / RS, dt, F32)
        sim.init_field(seed, k0, re_lambda)
        rec = {"t": [], "E": [], "eps": [], "derived": []}
        t = 0
        while True:
            E, eps = sim.stats()
            rec["t"].append(t)
            rec["E"].append(E)
            rec["eps"].append(eps)
            if t % derived_every == 0:
                d = sim.derived_stats()
                d.pop("D")
                d["t"] = t
                rec["derived"].append(d)
            if t >= T:
                break
            sim.step(every * per)
            t += every
        rec["nu"] = sim.nu
        sim.close()
        out[name] = rec
    dE = max(abs(a / b - 1) for a, b in zip(out["lbe"]["E"], out["dugks"]["E"]))
    de = max(abs(a / b - 1) for a, b in zip(out["lbe"]["eps"], out["dugks"]["eps"]))
    return {"N": N, "Re_lambda": re_lambda, "time": T, "u_prime": U_PRIME, "k0": k0, "seed": seed,
            "max_rel_diff_E": dE, "max_rel_diff_eps": de, "schemes": out}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=128)
    ap.add_argument("--time", type=int, default=2000)
    ap.add_argument("--re", default="26.06,52.12,104.24")
    a = ap.parse_args()
    res = [history(a.N, float(r), a.time) for r in a.re.split(",")]
    print(json.dumps(res))


if __name__ == "__main__":
    main()
