"""Pins of the oracle's lattice, equilibrium and MRT algebra against closed
forms (Sec. II.A, Eqs. 4-8; Sec. II.B)."""
import itertools

import numpy as np
import pytest

RNG = np.random.default_rng(20160115)


def test_velocity_set_structure(orc):
    xi, w = orc.lattice()
    assert xi.shape == (19, 3)
    assert tuple(xi[0]) == (0, 0, 0)
    assert len({tuple(v) for v in xi}) == 19
    r2 = (xi ** 2).sum(1)
    assert np.all(r2[1:7] == 1) and np.all(r2[7:] == 2)
    # opposite velocities sit in adjacent slots (i, i+1), i odd
    for i in range(1, 19, 2):
        assert np.all(xi[i] == -xi[i + 1])
    np.testing.assert_allclose(w[0], 1 / 3)
    np.testing.assert_allclose(w[1:7], 1 / 18)
    np.testing.assert_allclose(w[7:], 1 / 36)


def test_quadrature_moments(orc):
    """sum W = 1, sum W xi_a xi_b = delta/3, 4th moment = (dd+dd+dd)/9,
    odd moments vanish: the isotropy D3Q19 needs for Eq. 4."""
    xi, w = orc.lattice()
    xi = xi.astype(float)
    assert abs(w.sum() - 1) < 1e-15
    np.testing.assert_allclose(np.einsum("i,ia->a", w, xi), 0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, xi, xi), np.eye(3) / 3, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib,ic->abc", w, xi, xi, xi), 0, atol=1e-16)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, xi, xi, xi, xi)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9
    np.testing.assert_allclose(m4, iso, atol=1e-16)


@pytest.mark.parametrize("trial", range(5))
def test_equilibrium_moments(orc, trial):
    """Eq. 7 reproduces delta-rho, rho0 u, the incompressible second moment
    delta-rho c_s^2 I + rho0 u u, and the contracted third moment
    sum xi_a |xi|^2 f_eq = 5/3 rho0 u_a."""
    xi, _ = orc.lattice()
    xi = xi.astype(float)
    drho = RNG.normal() * 1e-2
    u = RNG.normal(size=3) * 0.1
    f = orc.feq(drho, u)
    assert abs(f.sum() - drho) < 1e-16
    np.testing.assert_allclose(xi.T @ f, u, atol=1e-16)
    pi = np.einsum("i,ia,ib->ab", f, xi, xi)
    np.testing.assert_allclose(pi, drho / 3 * np.eye(3) + np.outer(u, u), atol=1e-16)
    q = np.einsum("i,ia,i->a", f, xi, (xi ** 2).sum(1))
    np.testing.assert_allclose(q, 5.0 / 3.0 * u, atol=1e-16)


def test_mrt_matrix_orthogonal_with_known_norms(orc):
    """M M^T is diagonal with the D3Q19 row norms; M is invertible."""
    M = orc.mrt_matrix()
    G = M @ M.T
    norms = np.array([19, 2394, 252, 10, 40, 10, 40, 10, 40, 36, 72, 12, 24, 4, 4, 4, 8, 8, 8],
                     dtype=float)
    np.testing.assert_allclose(np.diag(G), norms, rtol=0, atol=1e-12)
    off = G - np.diag(np.diag(G))
    assert np.abs(off).max() < 1e-12
    np.testing.assert_allclose(np.linalg.inv(M) @ M, np.eye(19), atol=1e-13)


def test_mrt_moment_rows_match_their_definitions(orc):
    """Rows 0, 3, 5, 7 are density and momentum; 13-15 the off-diagonal
    second moments; 9, 11 the traceless diagonal ones (Sec. II.B)."""
    xi, _ = orc.lattice()
    M = orc.mrt_matrix()
    x, y, z = xi.T.astype(float)
    np.testing.assert_array_equal(M[0], np.ones(19))
    np.testing.assert_array_equal(M[3], x)
    np.testing.assert_array_equal(M[5], y)
    np.testing.assert_array_equal(M[7], z)
    np.testing.assert_array_equal(M[13], x * y)
    np.testing.assert_array_equal(M[14], y * z)
    np.testing.assert_array_equal(M[15], x * z)
    np.testing.assert_array_equal(M[9], 2 * x * x - y * y - z * z)
    np.testing.assert_array_equal(M[11], y * y - z * z)


@pytest.mark.parametrize("trial", range(4))
def test_meq_consistent_with_projected_equilibrium(orc, trial):
    """m_eq_k = M_k . f_eq for every row whose equilibrium is fixed by the
    hydrodynamics: 0, 1, 3-9, 11, 13-18.  Row 9 catches the 3 p_xx factor;
    rows 4/6/8 the q_eq = -2/3 j identity."""
    drho = RNG.normal() * 1e-2
    j = RNG.normal(size=3) * 0.1
    M = orc.mrt_matrix()
    meq = orc.mrt_meq(drho, j)
    proj = M @ orc.feq(drho, j)
    rows = [0, 1, 3, 4, 5, 6, 7, 8, 9, 11, 13, 14, 15, 16, 17, 18]
    np.testing.assert_allclose(meq[rows], proj[rows], atol=1e-15)
    # rows 2, 10, 12 are the model's free choices (omega_eps = omega_xx = 0)
    assert meq[10] == 0 and meq[12] == 0
    assert abs(meq[2] - (-475 / 63) * (j @ j)) < 1e-15


@pytest.mark.parametrize("trial", range(4))
def test_free_equilibrium_rows_reduce_to_bgk(orc, trial):
    """Rows 2, 10, 12 (eps, 3 pi_xx, pi_ww) carry the free parameters.  For
    the D3Q19 quadrature, the projection of the BGK equilibrium is
    M_2 f_eq = 3 drho - (11/2) j^2 (weights 1/3, 1/18, 1/36 against the eps
    polynomial, which takes the values 12, -4, 1 on the rest, axis and
    diagonal velocities) and M_10 f_eq = -(1/2) M_9 f_eq, M_12 f_eq =
    -(1/2) M_11 f_eq.  With (omega_eps, omega_epsj, omega_xx) = (3, -11/2,
    -1/2) every one of the 19 equilibrium moments must therefore equal
    M f_eq: a wrong row, sign or factor in the parametrised rows fails."""
    drho = RNG.normal() * 1e-2
    j = RNG.normal(size=3) * 0.1
    M = orc.mrt_matrix()
    proj = M @ orc.feq(drho, j)
    meq = orc.mrt_meq(drho, j, omegas=(3.0, -5.5, -0.5))
    np.testing.assert_allclose(meq, proj, rtol=0, atol=2e-15)
    # the paper's parameters are the same rows with other coefficients
    paper = orc.mrt_meq(drho, j)
    np.testing.assert_array_equal(orc.mrt_meq(drho, j, omegas=(0.0, -475.0 / 63.0, 0.0)), paper)


def test_mrt_rates_reproduce_viscosity(orc):
    """s9 = dt/(3 nu + dt/2) (Sec. IV.A) inverts Eq. 23's nu = (1/s9 - 1/2)/3;
    conserved moments have zero rate."""
    for nu in [1.2395e-2, 2.479e-2, 0.05, 1e-3]:
        s = orc.mrt_rates(nu)
        assert abs((1 / s[9] - 0.5) / 3 - nu) < 1e-15
        assert s[9] == s[11] == s[13] == s[14] == s[15]
        assert s[0] == s[3] == s[5] == s[7] == 0
        np.testing.assert_allclose(s[[1, 2, 4, 10, 16]], [1.19, 1.4, 1.2, 1.4, 1.98])


@pytest.mark.parametrize("srate", [0.6, 1.0, 1.7])
def test_mrt_reduces_to_bgk(orc, srate):
    """With one rate s for every moment and m_eq = M f_eq the MRT collision is
    the textbook single-relaxation LBGK update f - s (f - f_eq)."""
    M = orc.mrt_matrix()
    for _ in range(3):
        drho = RNG.normal() * 1e-2
        u = RNG.normal(size=3) * 0.05
        feq = orc.feq(drho, u)
        f = feq + RNG.normal(size=19) * 1e-3
        # shift f so it carries the same conserved moments as feq
        _, j = orc.moments(f)
        d0, _ = orc.moments(f)
        fe = orc.feq(d0, j)
        meq = M @ fe
        s = np.full(19, srate)
        got = orc.mrt_collide(s, f, meq)
        np.testing.assert_allclose(got, f - srate * (f - fe), atol=1e-14)


def test_mrt_collision_conserves_mass_momentum(orc):
    xi, _ = orc.lattice()
    s = orc.mrt_rates(0.01)
    for _ in range(5):
        f = orc.feq(RNG.normal() * 1e-2, RNG.normal(size=3) * 0.1) + RNG.normal(size=19) * 1e-3
        d, j = orc.moments(f)
        fp = orc.mrt_collide(s, f, orc.mrt_meq(d, j))
        assert abs(fp.sum() - d) < 1e-15
        np.testing.assert_allclose(xi.T @ fp, j, atol=1e-15)


def test_lbe_streaming_is_a_shift(orc):
    """With S = 0 Eq. 21 is pure streaming: f_i moves by xi_i with periodic
    wrap, i.e. numpy.roll of each population."""
    xi, _ = orc.lattice()
    f = RNG.normal(size=(19, 5, 6, 7))
    out = orc.lbe_step(f, s=np.zeros(19))
    for i in range(19):
        ref = np.roll(f[i], shift=(xi[i, 2], xi[i, 1], xi[i, 0]), axis=(0, 1, 2))
        np.testing.assert_array_equal(out[i], ref)


def test_every_population_pair_is_adjacent_in_index_space(orc):
    xi, _ = orc.lattice()
    for i, j in itertools.combinations(range(19), 2):
        if np.all(xi[i] == -xi[j]) and i > 0:
            assert j == i + 1 and i % 2 == 1
