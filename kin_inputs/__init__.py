"""Seeded synthetic inputs for the LBE/DUGKS solvers and their oracle.

This module is the only code that both the CUDA path's tests and the FP64
oracle's tests draw inputs from.  It holds none of the schemes' arithmetic
(no equilibrium, collision, flux or statistics): it produces velocity fields
and raw random arrays from seeds, nothing else.

Random numbers come from one counter-based generator, splitmix64 (Steele,
Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
    mix64(z) = z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
               z ^= z >> 27; z *= 0x94D049BB133111EB; z ^ (z >> 31)
    the m-th output (m = 0, 1, ...) of a stream seeded with s is
    mix64(s + (m + 1) * 0x9E3779B97F4A7C15)   (all mod 2^64)
The CUDA library's own field initialiser implements the same definition
independently; a test checks that both produce the same field.

Initial field of Sec. III (Eq. 25), with the generator the paper leaves
unstated fixed as follows (grid N^3, spectrum peak k0, Mach number Ma):
  * modes n = (nx, ny, nz), signed integers, shell s(n) = floor(|n| + 1/2);
    a mode is excited iff 1 <= s(n) <= N/2 - 1 (so no Nyquist component);
  * the canonical half space H holds n with nz > 0, or nz = 0 and ny > 0, or
    nz = ny = 0 and nx > 0; u_hat(-n) = conj(u_hat(n)) for n in H;
  * for n in H and component c in {0, 1, 2}: counter
    m = ((kz * N + ky) * N + kx) * 3 + c with (kx, ky, kz) = n mod N; key =
    output 0 of the stream seeded with `seed`; uniforms
    U1 = unit(output 2m of the stream seeded with key),
    U2 = unit(output 2m + 1), unit(v) = ((v >> 11) + 0.5) * 2^-53;
    Box-Muller: g = sqrt(-2 ln U1) (cos 2 pi U2 + i sin 2 pi U2);
  * projection onto the plane normal to n: u_hat -= n (n . u_hat) / |n|^2;
  * each shell is rescaled so sum_{n in shell} |u_hat|^2 / 2 equals
    E_t(s) = s^4 exp(-2 s^2 / k0^2);
  * a global factor makes <u.u> = Ma^2, i.e. u' = sqrt(<u.u>/3) = Ma c_s with
    c_s = 1/sqrt(3) (Eq. 29);
  * u(x) = sum_n u_hat(n) exp(2 pi i n.x / N), x = 0..N-1 per axis.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64_output(seed, m):
    """m-th output (m >= 0) of the splitmix64 stream seeded with `seed`."""
    seed = np.asarray(seed, dtype=np.uint64)
    m = np.asarray(m, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(seed + (m + np.uint64(1)) * GAMMA)


def unit(v):
    """Map 64-bit outputs to doubles in the open interval (0, 1)."""
    v = np.asarray(v, dtype=np.uint64)
    return ((v >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def _signed(k, n):
    return np.where(k > n // 2, k - n, k)


def dhit_spectral(N: int, seed: int, k0: float, Ma: float):
    """Half-spectrum u_hat of the initial field, shape (3, N, N, N//2+1)
    indexed [c][kz][ky][kx], plus diagnostics.  See the module docstring."""
    if N < 4 or N % 2:
        raise ValueError("N must be even and >= 4")
    nh = N // 2 + 1
    kz = np.arange(N).reshape(N, 1, 1)
    ky = np.arange(N).reshape(1, N, 1)
    kx = np.arange(nh).reshape(1, 1, nh)
    sz, sy, sx = _signed(kz, N), _signed(ky, N), kx + 0 * kz  # kx <= N/2 stays non-negative
    sz = np.broadcast_to(sz, (N, N, nh))
    sy = np.broadcast_to(sy, (N, N, nh))
    sx = np.broadcast_to(sx, (N, N, nh))
    n2 = (sx * sx + sy * sy + sz * sz).astype(np.int64)
    shell = np.floor(np.sqrt(n2.astype(np.float64)) + 0.5).astype(np.int64)
    smax = N // 2 - 1
    active = (shell >= 1) & (shell <= smax)

    in_h = (sz > 0) | ((sz == 0) & (sy > 0)) | ((sz == 0) & (sy == 0) & (sx > 0))
    cx = np.where(in_h, sx, -sx) % N
    cy = np.where(in_h, sy, -sy) % N
    cz = np.where(in_h, sz, -sz) % N
    key = splitmix64_output(np.uint64(seed), 0)
    base = ((cz.astype(np.uint64) * np.uint64(N) + cy.astype(np.uint64)) * np.uint64(N)
            + cx.astype(np.uint64)) * np.uint64(3)
    uh = np.zeros((3, N, N, nh), dtype=np.complex128)
    for c in range(3):
        m = base + np.uint64(c)
        u1 = unit(splitmix64_output(key, np.uint64(2) * m))
        u2 = unit(splitmix64_output(key, np.uint64(2) * m + np.uint64(1)))
        r = np.sqrt(-2.0 * np.log(u1))
        g = r * (np.cos(2.0 * np.pi * u2) + 1j * np.sin(2.0 * np.pi * u2))
        uh[c] = np.where(in_h, g, np.conj(g))
    uh *= active[None]

    # projection normal to n
    n2s = np.where(n2 > 0, n2, 1).astype(np.float64)
    ndotu = sx * uh[0] + sy * uh[1] + sz * uh[2]
    uh[0] -= sx * ndotu / n2s
    uh[1] -= sy * ndotu / n2s
    uh[2] -= sz * ndotu / n2s

    # per-shell rescale; modes with 0 < kx < N/2 stand for themselves and -n
    mult = np.where((sx > 0) & (sx < N // 2), 2.0, 1.0)
    e_mode = 0.5 * np.sum(np.abs(uh) ** 2, axis=0) * mult
    e_shell = np.bincount(shell[active].ravel(), weights=e_mode[active].ravel(),
                          minlength=smax + 1)
    s = np.arange(smax + 1, dtype=np.float64)
    e_target = s ** 4 * np.exp(-2.0 * s * s / (k0 * k0))
    e_target[0] = 0.0
    scale = np.zeros(smax + 1)
    ok = e_shell > 0
    scale[ok] = np.sqrt(e_target[ok] / e_shell[ok])
    uh *= np.where(active, scale[np.where(active, shell, 0)], 0.0)[None]

    total = float(np.sum(e_target[1:]))
    g = math.sqrt(Ma * Ma / (2.0 * total))
    uh *= g
    e_final = e_target * g * g
    k2 = (2.0 * np.pi / N) ** 2 * n2
    omega = float(np.sum(k2 * 0.5 * np.sum(np.abs(uh) ** 2, axis=0) * mult))
    uu = float(np.sum(np.sum(np.abs(uh) ** 2, axis=0) * mult))
    info = {
        "shell_energy": e_final,           # E(s) for s = 0..N/2-1
        "omega": omega,                     # sum |k|^2 |u_hat|^2 / 2
        "u_prime": math.sqrt(uu / 3.0),     # Eq. 29
        "uu": uu,
    }
    return uh, info


def dhit_velocity(N: int, seed: int, k0: float, Ma: float, return_info: bool = False):
    """Initial velocity u0, shape (3, N, N, N) indexed [c][z][y][x], FP64."""
    uh, info = dhit_spectral(N, seed, k0, Ma)
    u = np.empty((3, N, N, N))
    for c in range(3):
        u[c] = np.fft.irfftn(uh[c], s=(N, N, N), axes=(0, 1, 2)) * float(N) ** 3
    if return_info:
        return u, info
    return u


def nu_from_re_lambda(u_prime: float, omega: float, re_lambda: float) -> float:
    """Viscosity giving Taylor-microscale Reynolds number re_lambda for a field
    with rms u' and Omega = sum |k|^2 E: Eqs. 26, 28 and 30 give
    lambda = u' sqrt(15 / (2 Omega)) independent of nu, so
    nu = u'^2 sqrt(15 / (2 Omega)) / Re_lambda."""
    return u_prime * u_prime * math.sqrt(15.0 / (2.0 * omega)) / re_lambda


def taylor_green(nx: int, ny: int, nz: int, U: float):
    """2-D Taylor-Green vortex u = U sin(kx) cos(ky), v = -U cos(kx) sin(ky),
    w = 0 with k = 2 pi / nx (nx == ny), uniform in z."""
    if nx != ny:
        raise ValueError("nx must equal ny")
    k = 2.0 * np.pi / nx
    x = np.arange(nx).reshape(1, 1, nx)
    y = np.arange(ny).reshape(1, ny, 1)
    u = np.zeros((3, nz, ny, nx))
    u[0] = U * np.sin(k * x) * np.cos(k * y)
    u[1] = -U * np.cos(k * x) * np.sin(k * y)
    return u


def shear_wave(ny: int, U: float, nx: int = 1, nz: int = 1):
    """Shear wave u_x = U sin(k y), k = 2 pi / ny."""
    k = 2.0 * np.pi / ny
    y = np.arange(ny).reshape(1, ny, 1)
    u = np.zeros((3, nz, ny, nx))
    u[0] = U * np.sin(k * y) + 0.0 * np.zeros((nz, ny, nx))
    return u


def uniform_velocity(nx: int, ny: int, nz: int, u0):
    u = np.zeros((3, nz, ny, nx))
    for c in range(3):
        u[c] = u0[c]
    return u


def random_velocity(nx: int, ny: int, nz: int, seed: int, amp: float = 0.05):
    """Smooth-free random velocity (independent normals per cell), for tests
    of local arithmetic.  Uses numpy's PCG64 seeded with `seed`."""
    rng = np.random.default_rng(seed)
    return amp * rng.standard_normal((3, nz, ny, nx))


def random_populations(nx: int, ny: int, nz: int, seed: int, amp: float = 1e-3):
    """Independent normal perturbations, shape (19, nz, ny, nx), to add to an
    equilibrium state so the non-equilibrium part is not zero."""
    rng = np.random.default_rng(seed)
    return amp * rng.standard_normal((19, nz, ny, nx))
