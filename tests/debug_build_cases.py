"""Small one-step parity cases run against the KIN_DEBUG build of libkin.

Run by tests/test_gpu_debug_build.py in a process of its own (a process loads
one build of the library).  Prints one JSON line: per case the normalised
error against the FP64 oracle, the debug status after it, and the guard
check.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import kin_inputs as ki  # noqa: E402
import oracle  # noqa: E402
import paper_1601_03815_gb300 as kin  # noqa: E402


def state(N, seed):
    u = ki.random_velocity(N, N, N, seed, 0.03)
    return oracle.equilibrium_field(u) + ki.random_populations(N, N, N, seed + 1, 2e-5)


def err(got, ref):
    scale = np.abs(ref).reshape(19, -1).max(axis=1)
    return float((np.abs(got - ref).reshape(19, -1).max(axis=1) / scale).max())


def main():
    kin.load(debug=True)
    oracle.build()
    out = {"debug_build": kin.debug_status()[0], "cases": []}
    for scheme, dt in (("lbe", 1.0), ("dugks", 0.5)):
        for storage in (kin.F64, kin.F32, kin.F16):
            for N in (2, 5, 12, 33):
                for ty in ((4, 8) if scheme == "dugks" and storage != kin.F64 else (0,)):
                    f0 = state(N, 40 + N)
                    sim = kin.Sim(N, kin.LBE_MRT if scheme == "lbe" else kin.DUGKS, 0.013, 0.1, dt, storage)
                    if ty:
                        sim.set_tuning(tile_y=ty, zchunk=3)
                    sim.set_f(f0)
                    f_in = sim.get_f()
                    sim.step(1)
                    got = sim.get_f()
                    guards = "ok"
                    try:
                        sim.check_guards()
                    except kin.KinError as exc:
                        guards = str(exc)
                    sim.close()
                    _, word = kin.debug_status(reset=True)
                    out["cases"].append({"scheme": scheme, "storage": storage, "N": N, "tile_y": ty,
                                         "err": err(got, oracle.step(scheme, f_in, 0.013, dt)),
                                         "debug_word": word, "guards": guards})
    # a mixed ensemble (the persistent kernel's tile and node loops)
    members, refs = [], []
    for k, (scheme, N) in enumerate((("lbe", 9), ("dugks", 12), ("dugks", 5), ("lbe", 4))):
        dt = 1.0 if scheme == "lbe" else 0.45
        sim = kin.Sim(N, kin.LBE_MRT if scheme == "lbe" else kin.DUGKS, 0.015, 0.1, dt, kin.F32)
        sim.set_f(state(N, 70 + k))
        f = sim.get_f()
        members.append(sim)
        refs.append(oracle.step(scheme, oracle.step(scheme, f, 0.015, dt), 0.015, dt))
    ens = kin.Ensemble(members)
    ens.set_tuning(tile_y=4, zchunk=3, lbe_block=64)
    ens.step(2)
    e = max(err(m.get_f(), r) for m, r in zip(members, refs))
    ens.close()
    for m in members:
        m.close()
    _, word = kin.debug_status(reset=True)
    out["cases"].append({"scheme": "ensemble", "storage": kin.F32, "N": 0, "tile_y": 4, "err": e,
                         "debug_word": word, "guards": "ok"})
    print(json.dumps(out))


if __name__ == "__main__":
    main()
