"""Long-run parity of the CUDA path with stored FP64 oracle histories.

The stored files under tests/golden/ were written by
tests/golden/make_oracle_histories.py, which calls only the oracle and the
seeded input generator.  Tolerance: E(t) and eps(t) within 1e-4 relative over
the run (FP32 storage against the FP64 oracle); spectrum shells holding more
than 1e-6 of the peak shell within 1e-3 relative.  Reported (test
properties): R_m(s) = max_t |s / s_oracle - 1| for s = E, eps (the paper's
maximum relative error, Sec. IV.C) and the first step at which either
exceeds the tolerance, if any.
"""
import os

import numpy as np
import pytest

import kin_inputs as ki

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    path = os.path.join(GOLDEN, name)
    header, rows = [], []
    with open(path) as fh:
        for line in fh:
            if line.startswith("#"):
                header.append(line)
            elif line.strip():
                rows.append(line.split())
    return header, rows


def _nu_from_header(header):
    for tok in header[0].split():
        if tok.startswith("nu="):
            return float(tok[3:])
    raise ValueError("no nu in header")


UNIT_ROUNDOFF = {1: 2.0 ** -11, 2: 2.0 ** -8}  # FP16, BF16


def _storage_bounds(u, n, N):
    """E and eps bounds for 2-byte storage after n steps (derivation in
    tests/test_gpu_precision.py): 10 u^2 n + 3 u sqrt(n / N^3) + 1e-4, and
    2.5 times that for eps."""
    e = 10.0 * u * u * n + 3.0 * u * (n / N ** 3) ** 0.5 + 1e-4
    return e, 2.5 * e


@pytest.mark.parametrize("storage", [0, 1, 2])
@pytest.mark.parametrize("scheme", ["lbe", "dugks"])
def test_history_128cubed_2000_steps(kin, scheme, storage, record_property):
    """128^3, k0 = 8, Ma = 0.1, Re_lambda = 25, 2000 steps: E and eps every 10
    steps against the FP64 oracle, and with FP32 storage E(k) every 200 steps;
    FP16 / BF16 storage within the bounds of their storage rounding."""
    hist_name = "oracle_c2_128_%s.txt" % scheme
    spec_name = "oracle_c2_128_%s_spectrum.txt" % scheme
    header, rows = _read(hist_name)
    _, srows = _read(spec_name)
    last = int(rows[-1][0])
    if last < 2000:
        pytest.skip("stored oracle history incomplete (%d steps)" % last)
    N = 128
    u, info = ki.dhit_velocity(N, 1200, 8.0, 0.1, return_info=True)
    nu = ki.nu_from_re_lambda(info["u_prime"], info["omega"], 25.0)
    assert abs(nu / _nu_from_header(header) - 1) < 1e-14
    dt = 1.0 if scheme == "lbe" else 0.5
    sim = kin.Sim(N, kin.LBE_MRT if scheme == "lbe" else kin.DUGKS, nu, 0.1, dt, storage)
    tol_e, tol_eps = (1e-4, 1e-4) if storage == 0 else _storage_bounds(UNIT_ROUNDOFF[storage], last, N)
    sim.set_velocity(u)
    ref = {int(r[0]): (float(r[1]), float(r[2])) for r in rows}
    sref = {int(r[0]): np.array([float(v) for v in r[1:]]) for r in srows}
    worst_e = worst_eps = worst_k = 0.0
    first_breach = None
    n = 0
    while n <= last:
        if n in sref and storage == 0:
            E, eps, Ek = sim.stats(spectrum=True)
            Eo = sref[n]
            sig = Eo > 1e-6 * Eo.max()
            worst_k = max(worst_k, float(np.max(np.abs(Ek[:len(Eo)][sig] / Eo[sig] - 1))))
        else:
            E, eps = sim.stats()
        Eo, eo = ref[n]
        worst_e = max(worst_e, abs(E / Eo - 1))
        worst_eps = max(worst_eps, abs(eps / eo - 1))
        if first_breach is None and (abs(E / Eo - 1) >= tol_e or abs(eps / eo - 1) >= tol_eps):
            first_breach = n
        if n < last:
            sim.step(10)
        n += 10
    sim.close()
    record_property("R_m_E", worst_e)
    record_property("R_m_eps", worst_eps)
    record_property("first_breach_step", first_breach)
    assert worst_e < tol_e and worst_eps < tol_eps, (worst_e, worst_eps, "first breach at step", first_breach)
    assert worst_k < 1e-3, worst_k


def test_lbe_256_history_and_blowup(kin):
    """The 256^3 bench field (k0 = 8, Ma = 0.15, Re_lambda = 70): the FP32 LBE run
    follows the stored FP64 oracle history while it is smooth and becomes
    non-finite at the same check as the oracle (a stability result of the
    MRT-LBE scheme on this under-resolved, high-Mach field; DUGKS stays
    stable on it)."""
    header, rows = _read("oracle_lbe_256_blowup.txt")
    nu = _nu_from_header(header)
    N = 256
    u, info = ki.dhit_velocity(N, 1300, 8.0, 0.15, return_info=True)
    assert abs(ki.nu_from_re_lambda(info["u_prime"], info["omega"], 70.0) / nu - 1) < 1e-14
    sim = kin.Sim(N, kin.LBE_MRT, nu, 0.15, 1.0, kin.F32)
    sim.set_velocity(u)
    del u
    step = 0
    blew = None
    for r in rows:
        n = int(r[0])
        sim.step(n - step)
        step = n
        try:
            E, eps = sim.stats()
            finite = True
        except kin.KinError as exc:
            assert exc.code == kin.KIN_ENONFINITE
            finite = False
        if n <= 65:
            Eo, eo = float(r[1]), float(r[2])
            assert finite and abs(E / Eo - 1) < 1e-4 and abs(eps / eo - 1) < 1e-4, (n, E, Eo)
        elif r[1] == "nonfinite":
            assert not finite
            blew = n
            break
        elif finite:
            assert E > 0.01  # the growth has started, as in the oracle
    assert blew == int(rows[-1][0])
    sim.close()
