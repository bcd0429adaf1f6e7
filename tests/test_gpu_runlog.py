"""The JSON-lines run log: one record per logged step at the stated cadences,
with the values kin_stats gives for the same states."""
import io
import json

import pytest

import kin_inputs as ki

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scheme,dt", [("lbe", 1.0), ("dugks", 0.5)])
def test_run_log_records(kin, scheme, dt):
    from paper_1601_03815_gb300.runlog import run_logged

    N = 16
    u = ki.dhit_velocity(N, 31, 4.0, 0.1)
    sc = kin.LBE_MRT if scheme == "lbe" else kin.DUGKS
    a, b = kin.Sim(N, sc, 0.02, 0.1, dt, kin.F32), kin.Sim(N, sc, 0.02, 0.1, dt, kin.F32)
    a.set_velocity(u)
    b.set_velocity(u)
    buf = io.StringIO()
    summary = run_logged(a, 23, buf, stats_every=5, spectrum_every=10)
    recs = [json.loads(line) for line in buf.getvalue().splitlines()]
    assert recs[0]["kind"] == "run" and recs[0]["scheme"] == scheme and recs[-1]["kind"] == "summary"
    stats = [r for r in recs if r["kind"] == "stats"]
    assert [r["step"] for r in stats] == [0, 5, 10, 15, 20, 23]
    assert [("Ek" in r) for r in stats] == [True, False, True, False, True, False]
    for r in stats:
        b.step(r["step"] - b.steps_taken)
        E, eps = b.stats()
        assert r["E"] == E and r["eps"] == eps
        assert r["t"] == pytest.approx(r["step"] * dt)
    assert summary["steps"] == 23 and summary["mlups"] > 0
    a.close()
    b.close()
