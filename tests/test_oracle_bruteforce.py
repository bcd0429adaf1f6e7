"""Brute-force pin of the oracle's time steps on tiny periodic boxes.

A second, deliberately naive implementation written straight from the paper:
it visits one cell (LBE) or one face (DUGKS) at a time with explicit
neighbour lookups, builds the MRT matrix from the row polynomials of
Sec. II.B and applies M^-1 through a linear solve per cell, and evaluates the
DUGKS interface distribution of Eqs. 13 and 15-18 population by population,
with the face moments summed over all 19 reconstructed values.  It shares
nothing with the oracle but the velocity order, which is part of the public
layout and is checked against it first.  A transposed operand, a wrong sign
or a misplaced neighbour in either implementation shows up as a mismatch far
above rounding.
"""
import itertools

import numpy as np
import pytest

# D3Q19 (Eq. 5) in the library's order: 0 at rest, then opposite pairs (2p+1, 2p+2)
PAIRS = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, -1, 0), (1, 0, 1), (1, 0, -1), (0, 1, 1), (0, 1, -1)]
XI = [(0, 0, 0)] + [v for p in PAIRS for v in (p, tuple(-c for c in p))]
W = [1.0 / 3.0] + [1.0 / 18.0] * 6 + [1.0 / 36.0] * 12

SHAPES = [(3, 3, 3), (4, 4, 4), (3, 4, 5)]


def m_row(k, v):
    """Row k of the transformation matrix of Sec. II.B at velocity v."""
    x, y, z = v
    r2 = x * x + y * y + z * z
    rows = [
        1,
        19 * r2 - 30,
        (21 * r2 * r2 - 53 * r2 + 24) / 2,
        x, (5 * r2 - 9) * x,
        y, (5 * r2 - 9) * y,
        z, (5 * r2 - 9) * z,
        3 * x * x - r2, (3 * r2 - 5) * (3 * x * x - r2),
        y * y - z * z, (3 * r2 - 5) * (y * y - z * z),
        x * y, y * z, x * z,
        (y * y - z * z) * x, (z * z - x * x) * y, (x * x - y * y) * z,
    ]
    return rows[k]


def feq_cell(drho, j):
    """Eq. 7 with rho0 = 1, RT = 1/3."""
    out = np.empty(19)
    j2 = j[0] ** 2 + j[1] ** 2 + j[2] ** 2
    for i, v in enumerate(XI):
        eu = v[0] * j[0] + v[1] * j[1] + v[2] * j[2]
        out[i] = W[i] * (drho + 3.0 * eu + 4.5 * eu * eu - 1.5 * j2)
    return out


def naive_lbe(f, nu):
    """One MRT-LBE step (Eq. 21) with the equilibrium moments and rates of
    Secs. II.B and IV.A, pushed to x + xi_i on the periodic box."""
    nz, ny, nx = f.shape[1:]
    M = np.array([[m_row(k, v) for v in XI] for k in range(19)], dtype=float)
    s9 = 1.0 / (3.0 * nu + 0.5)
    S = np.diag([0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2, s9, 1.4, s9, 1.4, s9, s9, s9, 1.98, 1.98, 1.98])
    out = np.empty_like(f)
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        fc = f[:, z, y, x]
        m = M @ fc
        d, jx, jy, jz = m[0], m[3], m[5], m[7]
        j2 = jx * jx + jy * jy + jz * jz
        meq = np.array([
            d, -11.0 * d + 19.0 * j2, -475.0 / 63.0 * j2,
            jx, -2.0 / 3.0 * jx, jy, -2.0 / 3.0 * jy, jz, -2.0 / 3.0 * jz,
            3.0 * (2.0 * jx * jx - (jy * jy + jz * jz)) / 3.0, 0.0,
            jy * jy - jz * jz, 0.0,
            jx * jy, jy * jz, jx * jz,
            0.0, 0.0, 0.0,
        ])
        post = fc - np.linalg.solve(M, S @ (m - meq))
        for i, (cx, cy, cz) in enumerate(XI):
            out[i, (z + cz) % nz, (y + cy) % ny, (x + cx) % nx] = post[i]
    return out


def naive_dugks(ft, nu, dt):
    """One DUGKS step: Eq. 19 per cell, Eqs. 13, 15-18 per face and population,
    Eq. 20 and Eq. 9 per cell."""
    nz, ny, nx = ft.shape[1:]
    tau, h = 3.0 * nu, 0.5 * dt
    fbp = np.empty_like(ft)
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        c = ft[:, z, y, x]
        drho = c.sum()
        j = [sum(XI[i][a] * c[i] for i in range(19)) for a in range(3)]
        fbp[:, z, y, x] = (2 * tau - h) / (2 * tau + dt) * c + 3 * h / (2 * tau + dt) * feq_cell(drho, j)

    def X(i, p):
        z, y, x = p
        return fbp[i, z % nz, y % ny, x % nx]

    def shift(p, a, s):
        q = list(p)
        q[2 - a] += s  # p is (z, y, x); axis a = 0 is x
        return tuple(q)

    flux_sum = np.zeros_like(ft)
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        L = (z, y, x)
        for a in range(3):
            R = shift(L, a, 1)
            fbar = np.empty(19)
            for i, v in enumerate(XI):
                # value at the face, then minus h xi . sigma (Eq. 13)
                mid = 0.5 * (X(i, L) + X(i, R))
                sigma = [0.0, 0.0, 0.0]
                sigma[a] = X(i, R) - X(i, L)
                for t in range(3):
                    if t != a:
                        gL = (X(i, shift(L, t, 1)) - X(i, shift(L, t, -1))) / 2.0
                        gR = (X(i, shift(R, t, 1)) - X(i, shift(R, t, -1))) / 2.0
                        sigma[t] = 0.5 * (gL + gR)
                fbar[i] = mid - h * (v[0] * sigma[0] + v[1] * sigma[1] + v[2] * sigma[2])
            drho = fbar.sum()
            jb = [sum(XI[i][b] * fbar[i] for i in range(19)) for b in range(3)]
            fface = 2 * tau / (2 * tau + h) * fbar + h / (2 * tau + h) * feq_cell(drho, jb)
            for i, v in enumerate(XI):
                F = v[a] * fface[i]
                flux_sum[(i,) + L] += F          # leaves L through its +a face
                Rw = (R[0] % nz, R[1] % ny, R[2] % nx)
                flux_sum[(i,) + Rw] -= F         # enters R through its -a face
    return 4.0 / 3.0 * fbp - 1.0 / 3.0 * ft - dt * flux_sum


def _state(orc, shape, seed):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    u = 0.05 * rng.standard_normal((3, nz, ny, nx))
    drho = 1e-2 * rng.standard_normal((nz, ny, nx))
    return orc.equilibrium_field(u, drho) + 1e-3 * rng.standard_normal((19, nz, ny, nx))


def test_velocity_order_matches_the_oracle(orc):
    xi, w = orc.lattice()
    np.testing.assert_array_equal(np.asarray(xi), np.array(XI))
    np.testing.assert_allclose(w, W, rtol=0, atol=1e-16)


@pytest.mark.parametrize("shape", SHAPES)
def test_lbe_step_equals_naive_per_cell_version(orc, shape):
    f = _state(orc, shape, 31)
    nu = 0.013
    ref = naive_lbe(f, nu)
    got = orc.step("lbe", f, nu, 1.0)
    assert np.abs(got - ref).max() < 1e-14 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dt", [0.5, 0.35355])
def test_dugks_step_equals_naive_per_face_version(orc, shape, dt):
    f = _state(orc, shape, 47)
    nu = 0.013
    ref = naive_dugks(f, nu, dt)
    got = orc.step("dugks", f, nu, dt)
    assert np.abs(got - ref).max() < 1e-14 * max(1.0, np.abs(ref).max())
