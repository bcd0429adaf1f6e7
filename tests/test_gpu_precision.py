"""Reduced-precision storage against the FP64 oracle: the 64^3 version of the
256^3 timing field (k0 = 8, Ma = 0.15, Re_lambda = 70), 1000 steps, E and eps
every 10 steps and E(k) every 200, f stored in FP32 / FP16 / BF16 with FP32
arithmetic.  Bounds are twice the errors measured on GB300 (max relative
error over the run; E(k) over shells holding more than 1e-6 of the peak):

            E          eps        E(k)
  LBE f32   3.2e-7     7.5e-7     5.2e-6
  LBE f16   6.1e-5     7.4e-5     3.1e-2
  LBE bf16  4.5e-3     4.3e-3     1.5      (high shells: storage noise)
  DUG f32   2.3e-5     2.5e-5     8.0e-5
  DUG f16   7.1e-5     6.3e-5     9.5e-3
  DUG bf16  5.1e-3     5.8e-3     4.7e-1
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BOUNDS = {
    ("lbe", "f32"): (1e-6, 2e-6, 2e-5),
    ("lbe", "f16"): (1.5e-4, 1.5e-4, 0.07),
    ("lbe", "bf16"): (1e-2, 1e-2, 3.0),
    ("dugks", "f32"): (1e-4, 1e-4, 2e-4),
    ("dugks", "f16"): (1.5e-4, 1.5e-4, 0.02),
    ("dugks", "bf16"): (1.2e-2, 1.2e-2, 1.0),
}


def _oracle(name):
    hist, spec = {}, {}
    with open(os.path.join(GOLDEN, name + ".txt")) as fh:
        for line in fh:
            if line.startswith("#"):
                continue
            t = line.split()
            hist[int(t[0])] = (float(t[1]), float(t[2]))
    with open(os.path.join(GOLDEN, name + "_spectrum.txt")) as fh:
        for line in fh:
            if line.startswith("#"):
                continue
            t = line.split()
            spec[int(t[0])] = np.array([float(v) for v in t[1:]])
    return {"hist": hist, "spec": spec}


@pytest.mark.parametrize("scheme", ["lbe", "dugks"])
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_storage_precision_against_oracle_64(kin, scheme, storage):
    from paper_1601_03815_gb300 import precision as P

    ref = _oracle("oracle_c3_64_%s" % scheme)
    assert max(ref["hist"]) == 1000
    sc = kin.LBE_MRT if scheme == "lbe" else kin.DUGKS
    run = P.run_history(64, sc, P.STORAGES[storage], steps=1000)
    assert run["nonfinite_at"] is None
    err = P.errors(run, ref)
    assert err["checks"] == 101
    bE, beps, bk = BOUNDS[(scheme, storage)]
    assert err["E"] < bE and err["eps"] < beps and err["Ek"] < bk, err
