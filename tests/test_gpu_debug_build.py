"""Memory-checker substitutes (compute-sanitizer is not available on this GPU
pool): the KIN_DEBUG build's index checks and the guard regions around the
state buffers.

The debug build's stencil kernels check every global offset and the
shared-memory slot and row indices they use; a failed check skips the access
and records the first failure instead of trapping.  The small one-step parity
cases (N = 2, 5, 12, 33; both schemes; FP64, FP32, FP16; DUGKS tiles of 4 and
8 rows) and a mixed ensemble run against it in a process of their own: every
check must pass, parity must hold at the usual tolerances, and no guard byte
may change.
"""
import json
import os
import subprocess
import sys

import pytest

import kin_inputs as ki

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = {3: 1e-12, 0: 1e-5, 1: 2e-3}


def test_debug_build_small_parity_cases():
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_build_cases.py")], capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["debug_build"] is True
    assert len(res["cases"]) > 30
    for c in res["cases"]:
        assert c["debug_word"] == 0, c
        assert c["guards"] == "ok", c
        assert c["err"] < TOL[c["storage"]], c


@pytest.mark.parametrize("scheme,dt", [("lbe", 1.0), ("dugks", 0.5)])
@pytest.mark.parametrize("storage", [3, 0, 1])
@pytest.mark.parametrize("N", [2, 5, 33])
def test_guards_hold_after_steps(kin, scheme, dt, storage, N):
    sim = kin.Sim(N, kin.LBE_MRT if scheme == "lbe" else kin.DUGKS, 0.013, 0.1, dt, storage)
    sim.set_velocity(ki.random_velocity(N, N, N, 5 + N, 0.03))
    sim.step(3)
    sim.stats()
    sim.check_guards()
    sim.close()


def test_guard_check_reports_a_changed_byte(kin):
    for buffer in (0, 1):
        for side in (0, 1):
            sim = kin.Sim(6, kin.DUGKS, 0.013, 0.1, 0.5)
            sim.step(1)
            sim.check_guards()
            sim.corrupt_guard(buffer, side)
            with pytest.raises(kin.KinError) as e:
                sim.check_guards()
            assert e.value.code == kin.KIN_EGUARD
            sim.close()


def test_release_build_reports_no_debug_checks(kin):
    is_debug, word = kin.debug_status()
    assert is_debug is False and word == 0
