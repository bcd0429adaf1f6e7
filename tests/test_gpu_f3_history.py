"""Decay histories of the second workload (Sec. IV.D, Re_lambda = 52.12 and
104.24) against stored FP64 oracle runs.

The stored files under tests/golden/ (oracle_f3_64_<scheme>_re<Re>.txt) were
written by `python tests/golden/make_oracle_histories.py f3 <scheme> <Re>`,
which calls only the oracle and the seeded input generator: a 64^3 box of the
paper's decay field (spectrum shape k^4 exp(-0.14 k^2), u' = 0.032, seed 1700),
nu from Re_lambda, 400 lattice time units (MRT-LBE dt = 1, DUGKS dt = 0.5),
E and eps every 10 time units.  Tolerance: 1e-4 relative on E(t) and eps(t)
(FP32 storage against the FP64 oracle), the history tolerance of the plain
workload; R_m(E), R_m(eps) (max_t |s / s_oracle - 1|, Sec. IV.C) and the
first time of a breach are recorded as test properties.
"""
import math
import os

import pytest

import kin_inputs as ki

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read(path):
    header, rows = [], []
    with open(path) as fh:
        for line in fh:
            (header if line.startswith("#") else rows).append(line)
    rows = [r.split() for r in rows if r.strip()]
    nu = next(float(t[3:]) for t in header[0].split() if t.startswith("nu="))
    return nu, rows


@pytest.mark.parametrize("scheme", ["lbe", "dugks"])
@pytest.mark.parametrize("re", [52.12, 104.24])
def test_f3_history_against_oracle(kin, scheme, re, record_property):
    nu_o, rows = _read(os.path.join(GOLDEN, "oracle_f3_64_%s_re%g.txt" % (scheme, re)))
    N, seed = 64, 1700
    k0, Ma = math.sqrt(2.0 / 0.14), 0.032 / math.sqrt(1.0 / 3.0)
    u, info = ki.dhit_velocity(N, seed, k0, Ma, return_info=True)
    nu = ki.nu_from_re_lambda(info["u_prime"], info["omega"], re)
    assert abs(nu / nu_o - 1) < 1e-14
    dt = 1.0 if scheme == "lbe" else 0.5
    per = int(round(1.0 / dt))
    sim = kin.Sim(N, kin.LBE_MRT if scheme == "lbe" else kin.DUGKS, nu, Ma, dt, kin.F32)
    sim.set_velocity(u)
    t_prev = 0
    worst_e = worst_eps = 0.0
    first_breach = None
    for r in rows:
        t = int(r[0])
        sim.step((t - t_prev) * per)
        t_prev = t
        E, eps = sim.stats()
        de, dp = abs(E / float(r[1]) - 1), abs(eps / float(r[2]) - 1)
        worst_e, worst_eps = max(worst_e, de), max(worst_eps, dp)
        if first_breach is None and max(de, dp) >= 1e-4:
            first_breach = t
    sim.close()
    record_property("R_m_E", worst_e)
    record_property("R_m_eps", worst_eps)
    record_property("first_breach_time", first_breach)
    assert t_prev == 400
    assert worst_e < 1e-4 and worst_eps < 1e-4, (worst_e, worst_eps, "first breach at time", first_breach)
