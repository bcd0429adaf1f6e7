"""Reduced-precision storage against the FP64 oracle: the 64^3 version of the
256^3 timing field (k0 = 8, Ma = 0.15, Re_lambda = 70), 1000 steps, E and eps
every 10 steps and E(k) every 200, f stored in FP32 / FP16 / BF16 with FP32
arithmetic.

FP32 storage is held to the history tolerance of the plain workload (E, eps
within 1e-4; E(k) within 1e-3 on shells holding more than 1e-6 of the peak).

FP16 and BF16 bounds follow from the storage rounding.  With unit roundoff u
(2^-11 for FP16, 2^-8 for BF16) every stored value carries an error of at
most u |f_i|; the velocity error of a cell, sum_i xi_i e_i, then has at most
|delta u|^2 <= u^2 (sum_i |xi_i| |f_i|)^2 <= 10 u^2 |u|^2 in energy (f_i is
dominated by the linear term 3 W_i xi_i . u, and 10 populations cross each
axis), so one step injects at most 10 u^2 E of noise energy.  Rounding errors
of different steps are independent, so their energies add: after n steps the
injected energy is at most 10 u^2 n E.  The part of the error linear in the
noise, <u . delta u>, averages over the N^3 cells and walks randomly over the
steps: 3 u sqrt(n / N^3) (three standard deviations).  Hence
    |E - E_oracle| / E <= 10 u^2 n + 3 u sqrt(n / N^3) + 1e-4,
the last term being the FP32-arithmetic allowance.  eps weighs the white
noise with the central-difference wavenumbers, <sum_a sin^2 k_a> = 3/2 for
white noise against about 0.6 for the flow (|k| near 2 pi k0 / N): 2.5 times
the energy bound.  E(k): the noise is white, so shell s receives the fraction
m_s / N^3 of it (m_s modes); shells holding at least ten times their noise
bound are compared, each within its noise bound plus 1e-3.
"""
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
UNIT_ROUNDOFF = {"f16": 2.0 ** -11, "bf16": 2.0 ** -8}
N, STEPS = 64, 1000


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


def shell_modes(n):
    """Number of integer wavevectors of the n^3 box in each shell floor(|k| + 1/2)."""
    k = np.fft.fftfreq(n, 1.0 / n)
    kk = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
    s = np.floor(kk + 0.5).astype(int).ravel()
    return np.bincount(s)


def storage_bounds(u, steps, n):
    e = 10 * u * u * steps + 3 * u * math.sqrt(steps / n ** 3) + 1e-4
    return e, 2.5 * e


@pytest.mark.parametrize("scheme", ["lbe", "dugks"])
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_storage_precision_against_oracle_64(kin, scheme, storage):
    from paper_1601_03815_gb300 import precision as P

    ref = _oracle("oracle_c3_64_%s" % scheme)
    assert max(ref["hist"]) == STEPS
    sc = kin.LBE_MRT if scheme == "lbe" else kin.DUGKS
    run = P.run_history(N, sc, P.STORAGES[storage], steps=STEPS)
    assert run["nonfinite_at"] is None
    if storage == "f32":
        err = P.errors(run, ref)
        assert err["checks"] == 101
        assert err["E"] < 1e-4 and err["eps"] < 1e-4 and err["Ek"] < 1e-3, err
        return
    u = UNIT_ROUNDOFF[storage]
    bE, beps = storage_bounds(u, STEPS, N)
    err = P.errors(run, ref)
    assert err["checks"] == 101
    assert err["E"] < bE and err["eps"] < beps, (err, bE, beps)
    m = shell_modes(N)
    E0 = ref["hist"][0][0]
    compared = 0
    for n, b in ref["spec"].items():
        a = run["spec"][n]
        k = min(len(a), len(b), len(m))
        noise = 10 * u * u * max(n, 1) * E0 * m[:k] / N ** 3
        sel = b[:k] >= 10 * noise
        compared += int(sel.sum())
        assert np.all(np.abs(a[:k][sel] - b[:k][sel]) <= noise[sel] + 1e-3 * b[:k][sel]), (n, storage)
    assert compared > 0
