"""Pins of the oracle's statistics (Eqs. 26-30), of the seeded initial field
(Eq. 25 with the generator recipe of kin_inputs) and of the paper's printed
parameters (Table I, Sec. IV.A)."""
import math
import os

import numpy as np
import pytest

import kin_inputs as ki

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden():
    vals = {}
    with open(os.path.join(GOLDEN, "paper_parameters.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = line.split()[:2]
            vals[key] = float(val)
    return vals


@pytest.mark.parametrize("N,m", [(16, 1), (16, 3), (24, 5)])
def test_single_mode_energy_dissipation_spectrum(orc, N, m):
    """u_y = U sin(k x), k = 2 pi m / N: E = U^2/4, the spectrum holds U^2/4 in
    shell m, Omega = k^2 U^2/4, and the central-difference dissipation is
    2 nu <s_ab s_ab> = nu U^2 sin^2(k) / 2 (modified wavenumber sin k)."""
    U, nu = 0.03, 0.011
    k = 2 * np.pi * m / N
    x = np.arange(N)
    u = np.zeros((3, N, N, N))
    u[1] = U * np.sin(k * x)[None, None, :]
    E, eps = orc.energy_dissipation(u, nu)
    assert abs(E - U * U / 4) < 1e-17
    assert abs(eps - nu * U * U * np.sin(k) ** 2 / 2) < 1e-17
    Ek, omega = orc.spectrum(u)
    assert abs(Ek[m] - U * U / 4) < 1e-17
    assert abs(Ek.sum() - U * U / 4) < 1e-17
    assert abs(omega - k * k * U * U / 4) < 1e-16


def test_macro_inverts_equilibrium(orc):
    u = ki.random_velocity(5, 6, 7, 4)
    drho = 1e-2 * np.random.default_rng(5).standard_normal((7, 6, 5))
    f = orc.equilibrium_field(u, drho)
    d, uu = orc.macro(f)
    np.testing.assert_allclose(d, drho, atol=1e-16)
    np.testing.assert_allclose(uu, u, atol=1e-16)


def test_parseval(orc):
    u = ki.random_velocity(8, 10, 6, 9)
    Ek, _ = orc.spectrum(u)
    E, _ = orc.energy_dissipation(u, 0.01)
    assert abs(Ek.sum() - E) < 1e-14 * E


@pytest.mark.parametrize("N,k0,Ma", [(16, 4.0, 0.1), (32, 4.0, 0.1), (32, 8.0, 0.15)])
def test_initial_field_recipe(orc, N, k0, Ma):
    """The generated field is solenoidal, has u' = Ma c_s (Eq. 29) and its
    oracle-measured shell spectrum equals the prescribed k^4 exp(-2k^2/k0^2)
    shape times one global factor."""
    u, info = ki.dhit_velocity(N, 1234, k0, Ma, return_info=True)
    uh = np.fft.fftn(u, axes=(1, 2, 3))
    k = np.fft.fftfreq(N, 1.0 / N)
    div = k[None, None, :] * uh[0] + k[None, :, None] * uh[1] + k[:, None, None] * uh[2]
    assert np.abs(div).max() < 1e-12 * np.abs(uh).max()
    uprime = math.sqrt((u ** 2).sum(0).mean() / 3)
    assert abs(uprime - Ma / math.sqrt(3)) < 1e-14
    Ek, omega = orc.spectrum(u, N // 2)
    s = np.arange(N // 2, dtype=float)
    shape = s ** 4 * np.exp(-2 * s * s / k0 ** 2)
    g = Ek[1:].sum() / shape[1:].sum()
    np.testing.assert_allclose(Ek[1:], g * shape[1:], rtol=1e-10, atol=1e-30)
    assert Ek[0] < 1e-30
    assert abs(omega / info["omega"] - 1) < 1e-12
    assert abs(Ek.sum() - 1.5 * uprime ** 2) < 1e-14  # K = 3/2 u'^2


def test_viscosity_from_re_lambda(orc):
    """nu chosen from Re_lambda reproduces Re_lambda = u' lambda / nu with
    lambda = sqrt(15 nu / eps) u' and eps = 2 nu Omega (Eqs. 26, 28, 30),
    Omega measured by the oracle's spectrum."""
    u, info = ki.dhit_velocity(32, 77, 4.0, 0.1, return_info=True)
    nu = ki.nu_from_re_lambda(info["u_prime"], info["omega"], 25.0)
    _, omega = orc.spectrum(u)
    eps = 2 * nu * omega
    lam = math.sqrt(15 * nu / eps) * info["u_prime"]
    assert abs(info["u_prime"] * lam / nu - 25.0) < 1e-10


def test_generator_is_seed_deterministic_and_seed_sensitive():
    a = ki.dhit_velocity(16, 5, 4.0, 0.1)
    b = ki.dhit_velocity(16, 5, 4.0, 0.1)
    c = ki.dhit_velocity(16, 6, 4.0, 0.1)
    np.testing.assert_array_equal(a, b)
    assert np.abs(a - c).max() > 1e-3


def test_splitmix64_reference_values():
    """splitmix64 stream seeded with 0: published first outputs."""
    out = [int(ki.splitmix64_output(np.uint64(0), m)) for m in range(3)]
    assert out == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_paper_parameters_are_consistent(orc):
    """Relations among the printed parameters (Sec. IV.A, Table I)."""
    g = _golden()
    # Ma_max = |u|_max / c_s with c_s^2 = RT = 1/3
    assert abs(g["u_max_lattice"] * math.sqrt(3) - g["Ma_max"]) < 1e-4
    # K0 = 3/2 u'^2 in both unit systems
    assert abs(math.sqrt(g["K0_lattice"] / 1.5) - g["u_prime0_lattice"]) < 5e-5
    assert abs(math.sqrt(g["K0_ps"] / 1.5) - g["u_prime0_ps"]) < 5e-5
    # velocity scale V_s: lattice velocity = V_s * spectral velocity
    vs = math.sqrt(g["K0_lattice"] / g["K0_ps"])
    assert abs(vs - g["V_s"]) < 5e-5
    # nu_lattice = nu_ps * V_s * N / (2 pi) for both grids (L = 2 pi vs L = N)
    for N, key in [(128, "nu_lbe_128"), (256, "nu_lbe_256")]:
        assert abs(g["nu_ps"] * vs * N / (2 * math.pi) / g[key] - 1) < 2e-3
    # DUGKS time step from the CFL rule dt = gamma dx / (sqrt(2) c)
    assert abs(g["gamma_cfl"] / math.sqrt(2) - g["dt_dugks"]) < 1e-4
    # the oracle's rates carry the printed values
    s = orc.mrt_rates(g["nu_lbe_128"])
    np.testing.assert_allclose(s[[1, 2, 4, 10, 16]],
                               [g["s1"], g["s2"], g["s4"], g["s10"], g["s16"]])
    M = orc.mrt_matrix()
    j = np.array([0.01, 0.02, -0.03])
    assert abs(orc.mrt_meq(0.0, j)[2] - g["omega_epsj"] * (j @ j)) < 1e-9
    # per-iteration costs: LBE about 36.8 % faster per step
    assert abs(g["dugks_seconds_per_iteration_128"] / g["lbe_seconds_per_iteration_128"] - 1.368) < 1e-3
