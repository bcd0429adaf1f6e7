"""Derived statistics on the GPU (kin_derived_stats: u', spectral eps,
lambda, Re_lambda, eta, D(k), velocity-derivative skewness and flatness)
against the oracle and against closed forms."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KEYS = ("E", "uprime", "eps", "lambda", "Re_lambda", "eta", "F")


@pytest.mark.parametrize("storage", [3, 0])
def test_derived_stats_match_oracle(kin, orc, storage):
    N = 32
    sim = kin.Sim(N, kin.DUGKS, 0.01, 0.1, 0.5, storage)
    sim.init_field(21, 4.0, 30.0)
    sim.step(5)
    d = sim.derived_stats()
    _, u = orc.macro(sim.get_f())
    ref = orc.derived_stats(u, sim.nu, kin.num_shells(N))
    for k in KEYS:
        assert d[k] == pytest.approx(ref[k], rel=1e-10), k
    assert abs(d["S"] - ref["S"]) < 1e-9 * max(1.0, abs(ref["S"]))
    np.testing.assert_allclose(d["D"], ref["D"], rtol=1e-9, atol=1e-13 * ref["D"].max())
    # the state is untouched and the result reproducible
    d2 = sim.derived_stats()
    assert d2["S"] == d["S"] and d2["F"] == d["F"]
    sim.close()


def test_initial_field_has_the_requested_re_lambda(kin):
    sim = kin.Sim(48, kin.LBE_MRT, 0.01, 0.1, 1.0, kin.F64)
    sim.init_field(5, 6.0, 55.0)
    assert sim.derived_stats()["Re_lambda"] == pytest.approx(55.0, rel=1e-10)
    sim.close()


def test_two_mode_skewness_and_flatness_closed_form(kin):
    """u = A sin(kx) + B sin(2kx), v = C sin(ky), w = 0 through set_velocity:
    du/dx = a cos t + b cos 2t has <.^2> = (a^2 + b^2)/2, <.^3> = 3 a^2 b / 4,
    <.^4> = 3/8 a^4 + 3/2 a^2 b^2 + 3/8 b^4."""
    N, m = 32, 2
    A, B, C = 0.01, 0.004, 0.007
    k = 2 * np.pi * m / N
    x = np.arange(N)
    u = np.zeros((3, N, N, N))
    u[0] = (A * np.sin(k * x) + B * np.sin(2 * k * x))[None, None, :]
    u[1] = (C * np.sin(k * x))[None, :, None]
    sim = kin.Sim(N, kin.LBE_MRT, 0.02, 0.1, 1.0, kin.F64)
    sim.set_velocity(u)
    d = sim.derived_stats()
    a, b, c = A * k, 2 * B * k, C * k
    m2u, m3u = (a * a + b * b) / 2, 0.75 * a * a * b
    m4u = 3 / 8 * a ** 4 + 1.5 * a * a * b * b + 3 / 8 * b ** 4
    m2v, m4v = c * c / 2, 3 / 8 * c ** 4
    assert d["S"] == pytest.approx(m3u / (m2u ** 1.5 + m2v ** 1.5), rel=1e-10)
    assert d["F"] == pytest.approx((m4u + m4v) / (m2u ** 2 + m2v ** 2), rel=1e-10)
    sim.close()
