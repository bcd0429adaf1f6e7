"""FP64 CPU oracle for the LBE (MRT, D3Q19) and DUGKS steps of Wang, Wang & Guo,
"Comparison of the LBE and DUGKS methods for DNS of decaying homogeneous
isotropic turbulence" (arXiv:1601.03815).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline and reference legs of ``bench.py`` may import this package.  The product library
(``paper_1601_03815_gb300``) never imports it, and it never imports the product.

The time steppers live in ``kin_oracle.c`` (plain C, FP64, OpenMP); this module
marshals numpy arrays into it and adds the energy spectrum of Eq. 27, computed
with numpy's FFT as a library step.

Array layout: f has shape (19, nz, ny, nx) (x fastest), u has shape
(3, nz, ny, nx).  Population order is :func:`lattice`.

Parity status: see the header of ``kin_oracle.h``.  ``spectrum`` is pinned by
single-mode closed forms and Parseval (tests/test_oracle_stats.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kin_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

Q = 19
RHO0 = 1.0  # reference density (lattice units, Sec. IV.A)


def build(force: bool = False) -> str:
    """Compile kin_oracle.c into liboracle.so beside it (gcc, -O2, OpenMP)."""
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(_SRC),
                                             os.path.getmtime(os.path.join(_HERE, "kin_oracle.h")))):
        return _SO
    tmp = _SO + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            d = ctypes.c_double
            i = ctypes.c_int
            p = ctypes.c_void_p
            lib.orc_lattice.argtypes = [p, p]
            lib.orc_feq.argtypes = [d, d, d, d, p]
            lib.orc_moments.argtypes = [p, p, p]
            lib.orc_mrt_matrix.argtypes = [p]
            lib.orc_mrt_meq.argtypes = [d, d, d, d, p]
            lib.orc_mrt_meq_w.argtypes = [d, d, d, d, d, d, d, p]
            lib.orc_mrt_rates.argtypes = [d, p]
            lib.orc_mrt_collide.argtypes = [p, p, p, p]
            lib.orc_lbe_step.argtypes = [i, i, i, p, p, p]
            lib.orc_lbe_step.restype = i
            lib.orc_lbe_consistent_step.argtypes = [i, i, i, p, p, p, p]
            lib.orc_lbe_consistent_step.restype = i
            lib.orc_dugks_tau.argtypes = [d]
            lib.orc_dugks_tau.restype = d
            lib.orc_dugks_prestep_cell.argtypes = [d, d, p, p, p]
            lib.orc_dugks_step.argtypes = [i, i, i, d, d, p, p]
            lib.orc_dugks_step.restype = i
            lib.orc_equilibrium_field.argtypes = [i, i, i, p, p, p]
            lib.orc_macro.argtypes = [i, i, i, p, p, p]
            lib.orc_energy_dissipation.argtypes = [i, i, i, d, p, p, p]
            lib.orc_num_threads.restype = i
            lib.orc_set_num_threads.argtypes = [i]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return _load().orc_num_threads()


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))


def lattice():
    """D3Q19 velocities xi (19, 3) int and weights W (19,) (Sec. II.A)."""
    xi = np.zeros(Q * 3, dtype=np.int32)
    w = np.zeros(Q, dtype=np.float64)
    _load().orc_lattice(_ptr(xi), _ptr(w))
    return xi.reshape(Q, 3).astype(np.int64), w


def feq(drho: float, u) -> np.ndarray:
    """Discrete equilibrium of Eq. 7 for one cell."""
    out = np.zeros(Q)
    _load().orc_feq(float(drho), float(u[0]), float(u[1]), float(u[2]), _ptr(out))
    return out


def moments(f) -> tuple[float, np.ndarray]:
    f = _f64(f)
    r = np.zeros(1)
    j = np.zeros(3)
    _load().orc_moments(_ptr(f), _ptr(r), _ptr(j))
    return float(r[0]), j


def mrt_matrix() -> np.ndarray:
    M = np.zeros(Q * Q)
    _load().orc_mrt_matrix(_ptr(M))
    return M.reshape(Q, Q)


def mrt_meq(drho: float, j, omegas=None) -> np.ndarray:
    """Sec. II.B equilibrium moments; omegas = (omega_eps, omega_epsj,
    omega_xx), default the paper's (0, -475/63, 0)."""
    out = np.zeros(Q)
    if omegas is None:
        _load().orc_mrt_meq(float(drho), float(j[0]), float(j[1]), float(j[2]), _ptr(out))
    else:
        w = [float(v) for v in omegas]
        _load().orc_mrt_meq_w(float(drho), float(j[0]), float(j[1]), float(j[2]), w[0], w[1], w[2], _ptr(out))
    return out


def mrt_rates(nu: float) -> np.ndarray:
    s = np.zeros(Q)
    _load().orc_mrt_rates(float(nu), _ptr(s))
    return s


def mrt_collide(s, f, meq) -> np.ndarray:
    s, f, meq = _f64(s), _f64(f), _f64(meq)
    out = np.zeros(Q)
    _load().orc_mrt_collide(_ptr(s), _ptr(f), _ptr(meq), _ptr(out))
    return out


def _dims(f: np.ndarray):
    if f.ndim != 4 or f.shape[0] != Q:
        raise ValueError("f must have shape (19, nz, ny, nx)")
    nz, ny, nx = f.shape[1:]
    return nx, ny, nz


def lbe_step(f, nu: float | None = None, s=None) -> np.ndarray:
    """One MRT-LBE step (Eq. 21) with the Sec. IV.A rates for viscosity nu, or
    with an explicit rate vector s."""
    f = _f64(f)
    nx, ny, nz = _dims(f)
    if s is None:
        s = mrt_rates(nu)
    s = _f64(s)
    out = np.empty_like(f)
    rc = _load().orc_lbe_step(nx, ny, nz, _ptr(s), _ptr(f), _ptr(out))
    if rc != 0:
        raise RuntimeError("orc_lbe_step failed: %d" % rc)
    return out


def lbe_consistent_step(f, u0, nu: float) -> np.ndarray:
    """One iteration of the consistent initialisation (Sec. IV.A, after Mei
    et al.): the MRT-LBE step with the velocity held at u0 (3, nz, ny, nx)."""
    f = _f64(f)
    nx, ny, nz = _dims(f)
    u0 = _f64(u0)
    if u0.shape != (3, nz, ny, nx):
        raise ValueError("u0 must have shape (3, nz, ny, nx)")
    s = _f64(mrt_rates(nu))
    out = np.empty_like(f)
    rc = _load().orc_lbe_consistent_step(nx, ny, nz, _ptr(s), _ptr(u0), _ptr(f), _ptr(out))
    if rc != 0:
        raise RuntimeError("orc_lbe_consistent_step failed: %d" % rc)
    return out


def lbe_consistent(u0, nu: float, iters: int, drho0=None):
    """The consistent initial distributions for the velocity u0: iterate
    lbe_consistent_step from f_eq(drho0, u0) (drho0 = 0 by default) `iters`
    times.  Returns (f, residuals) with residuals[k] = max |drho^{k+1} -
    drho^k| over the box."""
    u0 = _f64(u0)
    f = equilibrium_field(u0, drho0)
    res = []
    d_prev = f.sum(axis=0)
    for _ in range(iters):
        f = lbe_consistent_step(f, u0, nu)
        d = f.sum(axis=0)
        res.append(float(np.abs(d - d_prev).max()))
        d_prev = d
    return f, res


def dugks_consistent_step(f, u0, nu: float, dt: float) -> np.ndarray:
    """One iteration of the consistent initialisation for DUGKS (Sec. IV.A
    applies the procedure of Mei et al. to both schemes): the DUGKS step of
    Eqs. 9-20, after which the momentum of the new f-tilde is set back to
    rho0 u0 along the linear term of the equilibrium (Eq. 7),
    f-tilde_i += 3 W_i xi_i . rho0 (u0 - u), which changes neither the mass
    nor the second moment.  The density evolves freely."""
    xi, w = lattice()
    u0 = _f64(u0)
    g = dugks_step(f, nu, dt)
    _, u = macro(g)
    du = RHO0 * (u0 - u)
    g += 3.0 * w[:, None, None, None] * np.einsum("ia,azyx->izyx", xi.astype(np.float64), du)
    return g


def dugks_consistent(u0, nu: float, dt: float, iters: int, drho0=None):
    """The consistent initial distributions for DUGKS: iterate
    dugks_consistent_step from f_eq(drho0, u0) `iters` times.  Returns
    (f, residuals), residuals[k] = max |drho^{k+1} - drho^k|."""
    u0 = _f64(u0)
    f = equilibrium_field(u0, drho0)
    res = []
    d_prev = f.sum(axis=0)
    for _ in range(iters):
        f = dugks_consistent_step(f, u0, nu, dt)
        d = f.sum(axis=0)
        res.append(float(np.abs(d - d_prev).max()))
        d_prev = d
    return f, res


def dugks_tau(nu: float) -> float:
    return _load().orc_dugks_tau(float(nu))


def dugks_prestep_cell(tau: float, dt: float, ft):
    ft = _f64(ft)
    b = np.zeros(Q)
    p = np.zeros(Q)
    _load().orc_dugks_prestep_cell(float(tau), float(dt), _ptr(ft), _ptr(b), _ptr(p))
    return b, p


def dugks_step(f, nu: float, dt: float) -> np.ndarray:
    """One DUGKS step (Eqs. 9-20) on the stored f-tilde."""
    f = _f64(f)
    nx, ny, nz = _dims(f)
    out = np.empty_like(f)
    rc = _load().orc_dugks_step(nx, ny, nz, float(nu), float(dt), _ptr(f), _ptr(out))
    if rc != 0:
        raise RuntimeError("orc_dugks_step failed: %d" % rc)
    return out


def step(scheme: str, f, nu: float, dt: float) -> np.ndarray:
    if scheme == "lbe":
        return lbe_step(f, nu)
    if scheme == "dugks":
        return dugks_step(f, nu, dt)
    raise ValueError(scheme)


def equilibrium_field(u, drho=None) -> np.ndarray:
    """f = f_eq(drho, u) everywhere (Eq. 7); u has shape (3, nz, ny, nx)."""
    u = _f64(u)
    nz, ny, nx = u.shape[1:]
    f = np.empty((Q, nz, ny, nx))
    d = None if drho is None else _f64(drho)
    _load().orc_equilibrium_field(nx, ny, nz, None if d is None else _ptr(d), _ptr(u), _ptr(f))
    return f


def macro(f):
    """delta-rho (nz, ny, nx) and u (3, nz, ny, nx) from f (Eq. 8)."""
    f = _f64(f)
    nx, ny, nz = _dims(f)
    drho = np.empty((nz, ny, nx))
    u = np.empty((3, nz, ny, nx))
    _load().orc_macro(nx, ny, nz, _ptr(f), _ptr(drho), _ptr(u))
    return drho, u


def energy_dissipation(u, nu: float):
    """E = <u.u>/2 and eps = 2 nu <s_ab s_ab> (central differences)."""
    u = _f64(u)
    nz, ny, nx = u.shape[1:]
    E = np.zeros(1)
    eps = np.zeros(1)
    _load().orc_energy_dissipation(nx, ny, nz, float(nu), _ptr(u), _ptr(E), _ptr(eps))
    return float(E[0]), float(eps[0])


def stats(f, nu: float):
    """(E, eps) of the state f."""
    _, u = macro(f)
    return energy_dissipation(u, nu)


def spectrum(u, nshell: int | None = None):
    """Energy spectrum of Eq. 27 summed over integer shells.

    u_hat(k) = N^-3 sum_x u(x) exp(-i k.x); mode n goes to shell
    floor(|n| + 1/2); E(s) = sum over the shell of |u_hat|^2 / 2.  Returns
    (E[0..nshell-1], Omega) where Omega = sum over all modes of
    |k|^2 |u_hat|^2 / 2 with k = 2 pi n / N, so eps_spectral = 2 nu Omega
    (Eq. 26).  The default nshell covers every mode (shells up to sqrt(3) N/2).
    """
    u = _f64(u)
    nz, ny, nx = u.shape[1:]
    ncell = nx * ny * nz
    uh = np.fft.fftn(u, axes=(1, 2, 3)) / ncell
    e = 0.5 * np.sum(np.abs(uh) ** 2, axis=0)
    kz = np.fft.fftfreq(nz, 1.0 / nz)
    ky = np.fft.fftfreq(ny, 1.0 / ny)
    kx = np.fft.fftfreq(nx, 1.0 / nx)
    n2 = kz[:, None, None] ** 2 + ky[None, :, None] ** 2 + kx[None, None, :] ** 2
    shell = np.floor(np.sqrt(n2) + 0.5).astype(np.int64)
    if nshell is None:
        nshell = int(shell.max()) + 1
    E = np.bincount(shell.ravel(), weights=e.ravel(), minlength=nshell)[:nshell]
    k2 = (2 * np.pi) ** 2 * (kz[:, None, None] ** 2 / nz ** 2 + ky[None, :, None] ** 2 / ny ** 2
                             + kx[None, None, :] ** 2 / nx ** 2)
    omega = float(np.sum(k2 * e))
    return E, omega


def derived_stats(u, nu: float, nshell: int | None = None):
    """Derived statistics of Sec. III: u', the Taylor microscale lambda,
    Re_lambda, the Kolmogorov length eta, the dissipation spectrum
    D(k) = 2 nu k^2 E(k), and the velocity-derivative skewness S and flatness F
    averaged over the three directions.

    eps is the spectral dissipation 2 nu sum_k |k|^2 E (Eq. 26); D(n) bins the
    same per-mode terms by shell, so sum_n D(n) = eps.  The derivatives
    du/dx, dv/dy, dw/dz are spectral (i k u_hat, Nyquist wavenumber dropped),
    taken with numpy's one-dimensional FFT along their own axis.

    S and F are the direction-summed third and fourth moments over the
    direction-summed powers of the second moment.  The printed formulas carry
    an extra factor 3 in the denominator, which would make a Gaussian field's
    flatness 1 rather than 3; the text calls them the skewness and flatness
    averaged over the three directions, so the factor is read as spurious.
    """
    u = _f64(u)
    nz, ny, nx = u.shape[1:]
    ncell = nx * ny * nz
    uh = np.fft.fftn(u, axes=(1, 2, 3)) / ncell
    e = 0.5 * np.sum(np.abs(uh) ** 2, axis=0)
    fz = np.fft.fftfreq(nz, 1.0 / nz)
    fy = np.fft.fftfreq(ny, 1.0 / ny)
    fx = np.fft.fftfreq(nx, 1.0 / nx)
    n2 = fz[:, None, None] ** 2 + fy[None, :, None] ** 2 + fx[None, None, :] ** 2
    shell = np.floor(np.sqrt(n2) + 0.5).astype(np.int64)
    if nshell is None:
        nshell = int(shell.max()) + 1
    k2 = (2 * np.pi) ** 2 * (fz[:, None, None] ** 2 / nz ** 2 + fy[None, :, None] ** 2 / ny ** 2
                             + fx[None, None, :] ** 2 / nx ** 2)
    D = 2.0 * nu * np.bincount(shell.ravel(), weights=(k2 * e).ravel(), minlength=nshell)[:nshell]
    eps = 2.0 * nu * float(np.sum(k2 * e))
    uu = float(np.mean(np.sum(u * u, axis=0)))
    uprime = np.sqrt(uu / 3.0)
    lam = np.sqrt(15.0 * nu / eps) * uprime
    m = np.zeros((3, 3))  # m[a][p - 2] = <(d_a u_a)^p>
    for a, axis in ((0, 3), (1, 2), (2, 1)):
        n = u.shape[axis]
        f = np.fft.fftfreq(n, 1.0 / n)
        k = 2.0 * np.pi * f / n
        if n % 2 == 0:
            k[n // 2] = 0.0  # the Nyquist wavenumber has no real derivative
        shape = [1, 1, 1]
        shape[axis - 1] = n
        d = np.real(np.fft.ifft(1j * k.reshape(shape) * np.fft.fft(u[a], axis=axis - 1), axis=axis - 1))
        for p in (2, 3, 4):
            m[a, p - 2] = float(np.mean(d ** p))
    S = m[:, 1].sum() / np.sum(m[:, 0] ** 1.5)
    F = m[:, 2].sum() / np.sum(m[:, 0] ** 2)
    return {"E": 0.5 * uu, "uprime": float(uprime), "eps": eps, "lambda": float(lam),
            "Re_lambda": float(uprime * lam / nu), "eta": float((nu ** 3 / eps) ** 0.25),
            "S": float(S), "F": float(F), "D": D, "moments": m}

