"""Maximum stable Taylor-microscale Reynolds number of MRT-LBE and DUGKS on a
fixed mesh (Sec. IV.E: the paper raises Re_lambda at 128^3, DUGKS at CFL 0.9,
until a code blows up, without regard to accuracy).

For each Re_lambda of an increasing list the seeded initial field (spectrum
shape k^4 exp(-0.14 k^2), i.e. k0 = sqrt(2 / 0.14), and u' = 0.032 as in
Table I) is set, nu follows from Re_lambda in closed form, and each scheme runs
`steps` steps with E checked every `every` steps; a run is unstable if E or
eps becomes non-finite.  DUGKS uses dt = gamma / sqrt(2) with the CFL number
gamma (0.9 by default).

    python -m paper_1601_03815_gb300.stability [--N 128 --steps 10000]

prints one JSON line with every run and the largest stable Re_lambda per
scheme.
"""
from __future__ import annotations

import argparse
import json
import math

from . import DUGKS, F32, KIN_ENONFINITE, LBE_MRT, KinError, Sim

RS = math.sqrt(1.0 / 3.0)  # lattice sound speed
K0 = math.sqrt(2.0 / 0.14)  # the shape k^4 exp(-2 k^2 / k0^2) of the generator
U_PRIME = 0.032
DEFAULT_RE = (26.06, 104.24, 417.0, 1668.0, 6672.0, 26060.0, 104240.0, 416960.0, 1667840.0)


def run_one(N: int, scheme: int, re_lambda: float, steps: int, every: int, seed: int, gamma: float):
    """(first non-finite check step or None, nu) of one run."""
    dt = 1.0 if scheme == LBE_MRT else gamma / math.sqrt(2.0)
    sim = Sim(N, scheme, 0.01, U_PRIME / RS, dt, F32)
    try:
        sim.init_field(seed, K0, re_lambda)
        nu = sim.nu
        n = 0
        while n < steps:
            sim.step(every)
            n += every
            try:
                sim.stats()
            except KinError as exc:
                if exc.code != KIN_ENONFINITE:
                    raise
                return n, nu
        return None, nu
    finally:
        sim.close()


def sweep(N: int = 128, re_list=DEFAULT_RE, steps: int = 10000, every: int = 50, seed: int = 1600,
          gamma: float = 0.9):
    runs = []
    best = {}
    for name, scheme in (("lbe", LBE_MRT), ("dugks", DUGKS)):
        best[name] = None
        for re in re_list:
            bad, nu = run_one(N, scheme, re, steps, every, seed, gamma)
            runs.append({"scheme": name, "Re_lambda": re, "nu": nu, "nonfinite_at_step": bad})
            if bad is None:
                best[name] = re
            else:
                break  # larger Re_lambda only lowers nu further
    return {"N": N, "steps": steps, "check_every": every, "u_prime": U_PRIME, "k0": K0,
            "dugks_cfl": gamma, "seed": seed, "runs": runs, "max_stable_re_lambda": best,
            "note": "the list stops at its last entry: a scheme stable there may be stable beyond it"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", type=int, default=128)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--every", type=int, default=50)
    ap.add_argument("--cfl", type=float, default=0.9)
    a = ap.parse_args()
    print(json.dumps(sweep(a.N, steps=a.steps, every=a.every, gamma=a.cfl)))


if __name__ == "__main__":
    main()
