"""The stability-sweep and decay-history runners on small boxes: structure of
their reports, the sweep's stop at the first failure, and agreement of the two
schemes' decay where both resolve the flow."""
import math

import pytest

pytestmark = pytest.mark.gpu


def test_stability_sweep_reports_every_run_until_the_first_failure(kin):
    from paper_1601_03815_gb300 import stability

    res = stability.sweep(N=16, re_list=(20.0, 40.0), steps=100, every=50)
    assert res["N"] == 16 and res["dugks_cfl"] == 0.9
    runs = res["runs"]
    for name in ("lbe", "dugks"):
        mine = [r for r in runs if r["scheme"] == name]
        assert mine and mine[0]["Re_lambda"] == 20.0
        # nu follows Re_lambda: halving it doubles Re_lambda
        if len(mine) == 2:
            assert mine[0]["nu"] / mine[1]["nu"] == pytest.approx(2.0, rel=1e-12)
        stable = [r["Re_lambda"] for r in mine if r["nonfinite_at_step"] is None]
        assert res["max_stable_re_lambda"][name] == (max(stable) if stable else None)


def test_decay_histories_of_the_two_schemes_agree_on_a_resolved_flow(kin):
    from paper_1601_03815_gb300 import histories

    # spectrum peak at |n| = 1.5 in a 32 box: ~5 cells per radian at the peak
    h = histories.history(N=32, re_lambda=10.0, T=100, every=10, derived_every=50, k0=1.5)
    lbe, dug = h["schemes"]["lbe"], h["schemes"]["dugks"]
    assert lbe["t"] == dug["t"] == list(range(0, 101, 10))
    assert lbe["E"][0] == pytest.approx(dug["E"][0], rel=1e-6)  # same initial field
    assert all(b < a for a, b in zip(lbe["E"], lbe["E"][1:]))  # decaying
    assert h["max_rel_diff_E"] < 0.03
    assert all(math.isfinite(d["S"]) and d["F"] > 0 for d in lbe["derived"] + dug["derived"])
