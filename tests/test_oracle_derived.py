"""Pins of the oracle's derived statistics (Sec. III: u', lambda, Re_lambda,
eta, D(k), velocity-derivative skewness S and flatness F) against closed forms
of one- and two-mode fields and the Gaussian value of the flatness."""
import numpy as np
import pytest

import kin_inputs as ki

N = 32


def _mode(axis, m, amp, n=N):
    """amp sin(2 pi m x_axis / n) as a (n, n, n) array, axis 0 = x."""
    x = np.arange(n)
    s = amp * np.sin(2 * np.pi * m * x / n)
    shape = [1, 1, 1]
    shape[2 - axis] = n
    return np.broadcast_to(s.reshape(shape), (n, n, n)).copy()


def test_single_mode_closed_forms(orc):
    A, m, nu = 0.01, 3, 0.02
    k = 2 * np.pi * m / N
    u = np.zeros((3, N, N, N))
    u[0] = _mode(0, m, A)
    d = orc.derived_stats(u, nu)
    assert abs(d["S"]) < 1e-12
    assert d["F"] == pytest.approx(1.5, rel=1e-12)  # <cos^4> / <cos^2>^2
    assert d["uprime"] == pytest.approx(A / np.sqrt(6), rel=1e-12)
    eps = 2 * nu * k * k * A * A / 4
    assert d["eps"] == pytest.approx(eps, rel=1e-12)
    assert d["lambda"] == pytest.approx(np.sqrt(5) / k, rel=1e-12)
    assert d["Re_lambda"] == pytest.approx(A / np.sqrt(6) * np.sqrt(5) / k / nu, rel=1e-12)
    assert d["eta"] == pytest.approx((nu ** 3 / eps) ** 0.25, rel=1e-12)
    D = d["D"]
    assert D[m] == pytest.approx(eps, rel=1e-12)
    assert np.abs(np.delete(D, m)).max() < 1e-12 * eps


def test_two_mode_skewness_and_flatness(orc):
    """u = A sin(kx) + B sin(2kx), v = C sin(ky), w = 0:
    du/dx = a cos t + b cos 2t (a = Ak, b = 2Bk) has <.^2> = (a^2 + b^2)/2,
    <.^3> = 3 a^2 b / 4, <.^4> = 3/8 a^4 + 3/2 a^2 b^2 + 3/8 b^4."""
    A, B, C, m = 0.01, 0.004, 0.007, 2
    k = 2 * np.pi * m / N
    u = np.zeros((3, N, N, N))
    u[0] = _mode(0, m, A) + _mode(0, 2 * m, B)
    u[1] = _mode(1, m, C)
    d = orc.derived_stats(u, 0.01)
    a, b, c = A * k, 2 * B * k, C * k
    m2u, m3u = (a * a + b * b) / 2, 0.75 * a * a * b
    m4u = 3 / 8 * a ** 4 + 1.5 * a * a * b * b + 3 / 8 * b ** 4
    m2v, m4v = c * c / 2, 3 / 8 * c ** 4
    np.testing.assert_allclose(d["moments"][0], [m2u, m3u, m4u], rtol=1e-11)
    np.testing.assert_allclose(d["moments"][1], [m2v, 0, m4v], rtol=1e-11, atol=1e-22)
    assert d["S"] == pytest.approx(m3u / (m2u ** 1.5 + m2v ** 1.5), rel=1e-11)
    assert d["F"] == pytest.approx((m4u + m4v) / (m2u ** 2 + m2v ** 2), rel=1e-11)


def test_gaussian_field_flatness_is_three(orc):
    """Random phases: the derivatives are Gaussian (F = 3, S = 0) up to
    sampling error."""
    u = ki.dhit_velocity(64, 7, 4.0, 0.1)
    d = orc.derived_stats(u, 0.01)
    assert abs(d["F"] - 3.0) < 0.15
    assert abs(d["S"]) < 0.05


def test_re_lambda_matches_the_viscosity_recipe(orc):
    """nu chosen for a target Re_lambda by the closed form of the input recipe
    gives back that Re_lambda."""
    u = ki.dhit_velocity(N, 11, 4.0, 0.1)
    uprime = np.sqrt(np.mean(np.sum(u * u, axis=0)) / 3)
    _, omega = orc.spectrum(u)
    nu = ki.nu_from_re_lambda(uprime, omega, 42.0)
    d = orc.derived_stats(u, nu)
    assert d["Re_lambda"] == pytest.approx(42.0, rel=1e-12)
    assert d["D"].sum() == pytest.approx(d["eps"], rel=1e-12)
