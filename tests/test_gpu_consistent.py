"""kin_init_consistent against the oracle's consistent initialisation
(Sec. IV.A, the iteration of Mei et al.): the same number of iterations from
the same state gives the same distributions, and converged on a Taylor-Green
vortex the density carries the pressure of the Poisson equation."""
import numpy as np
import pytest

import kin_inputs as ki

pytestmark = pytest.mark.gpu

NU = 0.05


def _err(got, ref):
    scale = np.abs(ref).reshape(19, -1).max(axis=1)
    return (np.abs(got - ref).reshape(19, -1).max(axis=1) / scale).max()


@pytest.mark.parametrize("storage,tol", [(3, 1e-12), (0, 1e-5)])
@pytest.mark.parametrize("N", [16, 15])
def test_iterations_match_the_oracle(kin, orc, storage, tol, N):
    u = ki.random_velocity(N, N, N, 900 + N, 0.03)
    sim = kin.Sim(N, kin.LBE_MRT, NU, 0.1, 1.0, storage)
    sim.set_velocity(u)
    iters, res = sim.init_consistent(40, -1.0)  # no early stop
    assert iters == 40 and res > 0.0
    ref, rres = orc.lbe_consistent(u, NU, 40)
    assert _err(sim.get_f(), ref) < tol
    assert abs(res / rres[-1] - 1) < 1e-3  # the same change of delta-rho in the last iteration
    assert sim.steps_taken == 0
    sim.step(2)
    E, eps = sim.stats()
    assert np.isfinite(E) and E > 0
    sim.close()


def test_converged_density_is_the_taylor_green_pressure(kin):
    N, U = 32, 0.02
    k = 2 * np.pi / N
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    u = np.zeros((3, N, N, N))
    u[0] = U * np.sin(k * x) * np.cos(k * y)
    u[1] = -U * np.cos(k * x) * np.sin(k * y)
    sim = kin.Sim(N, kin.LBE_MRT, NU, 0.1, 1.0, kin.F64)
    sim.set_velocity(u)
    iters, res = sim.init_consistent(4000, 1e-14)
    assert iters < 4000 and res <= 1e-14
    d = sim.get_f().sum(axis=0)
    exact = 0.75 * U ** 2 * (np.cos(2 * k * x) + np.cos(2 * k * y))
    assert abs(d.mean()) < 1e-17
    assert np.abs(d - exact).max() / np.abs(exact).max() < 1e-2
    sim.close()


@pytest.mark.parametrize("storage,tol", [(3, 1e-12), (0, 1e-5)])
@pytest.mark.parametrize("N", [16, 15])
def test_dugks_iterations_match_the_oracle(kin, orc, storage, tol, N):
    """DUGKS (Sec. IV.A applies the procedure to both schemes): a plain step
    and the momentum set back to rho0 u0, 40 iterations against the oracle."""
    dt = 0.5
    u = ki.random_velocity(N, N, N, 950 + N, 0.03)
    sim = kin.Sim(N, kin.DUGKS, NU, 0.1, dt, storage)
    sim.set_velocity(u)
    iters, res = sim.init_consistent(40, -1.0)
    assert iters == 40 and res > 0.0
    ref, rres = orc.dugks_consistent(u, NU, dt, 40)
    assert _err(sim.get_f(), ref) < tol
    assert abs(res / rres[-1] - 1) < 1e-3
    assert sim.steps_taken == 0
    sim.step(2)
    E, eps = sim.stats()
    assert np.isfinite(E) and E > 0
    sim.close()


def test_dugks_converged_density_is_the_taylor_green_pressure(kin):
    N, U = 32, 0.02
    k = 2 * np.pi / N
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    u = np.zeros((3, N, N, N))
    u[0] = U * np.sin(k * x) * np.cos(k * y)
    u[1] = -U * np.cos(k * x) * np.sin(k * y)
    sim = kin.Sim(N, kin.DUGKS, NU, 0.1, 0.5, kin.F64)
    sim.set_velocity(u)
    iters, res = sim.init_consistent(6000, 1e-14)
    assert iters < 6000 and res <= 1e-14
    f = sim.get_f()
    d = f.sum(axis=0)
    exact = 0.75 * U ** 2 * (np.cos(2 * k * x) + np.cos(2 * k * y))
    assert abs(d.mean()) < 1e-16
    assert np.abs(d - exact).max() / np.abs(exact).max() < 0.025
    sim.close()


def test_bad_arguments_are_rejected(kin):
    for scheme, dt in ((kin.LBE_MRT, 1.0), (kin.DUGKS, 0.5)):
        sim = kin.Sim(8, scheme, NU, 0.1, dt)
        with pytest.raises(kin.KinError) as e:
            sim.init_consistent(0)
        assert e.value.code == kin.KIN_EINVAL
        sim.close()


@pytest.mark.parametrize("scheme", ["lbe", "dugks"])
@pytest.mark.parametrize("storage,u_round", [(1, 2.0 ** -11), (2, 2.0 ** -8)])
def test_iterations_with_two_byte_storage(kin, orc, scheme, storage, u_round):
    """FP16 / BF16 storage: each iteration stores the state, rounding every
    value by at most u |f_i| (unit roundoff u).  The held momentum resets the
    rounding of j each iteration; the rest evolves slowly and its rounding
    errors add as a random walk, so after n iterations the distance to the
    FP64 oracle iteration stays within 4 sqrt(n) u of max |f_i| (four standard
    deviations of that walk, plus the initial rounding)."""
    N, n = 16, 40
    dt = 1.0 if scheme == "lbe" else 0.5
    u = ki.random_velocity(N, N, N, 970 + storage, 0.03)
    sim = kin.Sim(N, kin.LBE_MRT if scheme == "lbe" else kin.DUGKS, NU, 0.1, dt, storage)
    sim.set_velocity(u)
    iters, res = sim.init_consistent(n, -1.0)
    assert iters == n and np.isfinite(res)
    ref, _ = orc.lbe_consistent(u, NU, n) if scheme == "lbe" else orc.dugks_consistent(u, NU, dt, n)
    err = _err(sim.get_f(), ref)
    assert err < 4.0 * np.sqrt(n) * u_round, err
    sim.close()
