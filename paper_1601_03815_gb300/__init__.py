"""Python binding of libkin, the GB300 (sm_103a) CUDA library for the LBE and
DUGKS time steps of decaying homogeneous isotropic turbulence
(Wang, Wang & Guo, arXiv:1601.03815).

This module only marshals arguments to the C ABI declared in include/kin.h;
every step of the solver runs in the library's CUDA kernels.  There is no CPU
fallback: if libkin.so cannot be built or loaded, ``load()`` raises.

Host arrays are numpy FP64: f has shape (19, N, N, N) indexed [i][z][y][x],
u has shape (3, N, N, N).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

LBE_MRT = 0
DUGKS = 1
F32, F16, BF16, F64 = 0, 1, 2, 3
STORAGE_NAMES = {F32: "f32", F16: "f16", BF16: "bf16", F64: "f64"}
SCHEME_NAMES = {LBE_MRT: "lbe", DUGKS: "dugks"}

KIN_OK = 0
KIN_EINVAL = -1
KIN_ENOMEM = -2
KIN_ECUDA = -3
KIN_ENONFINITE = -4
KIN_ETIMEOUT = -5
KIN_ESTATE = -6
KIN_EGUARD = -7
KIN_EDEBUG = -8

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libkin.so")
DEBUG_LIB_PATH = os.path.join(_PKG, "libkin_debug.so")
_lib = None
_lock = threading.Lock()


class KinError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str):
        super().__init__("%s failed: %s (%d): %s" % (where, _strerror(code), code, detail))
        self.code = code


def _strerror(code: int) -> str:
    if _lib is None:
        return str(code)
    return _lib.kin_strerror(code).decode()


def _out2(out):
    """Pointer to a float64 C-contiguous array of at least 2 elements."""
    if not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous
            and out.size >= 2):
        raise ValueError("out must be a C-contiguous float64 array of at least 2 elements")
    return out.ctypes.data_as(ctypes.c_void_p)


def _declare(lib):
    c_int, c_double, c_void_p, c_size_t = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
    c_i64, c_u64 = ctypes.c_int64, ctypes.c_uint64
    P = ctypes.c_void_p
    sig = {
        "kin_lattice": (c_int, [P, P]),
        "kin_footprint_bytes": (c_size_t, [c_int, c_int, c_int]),
        "kin_create": (c_int, [c_int, c_int, c_double, c_double, c_double, c_int, c_void_p, P]),
        "kin_init_field": (c_int, [P, c_u64, c_double, c_double]),
        "kin_set_velocity": (c_int, [P, P]),
        "kin_set_f": (c_int, [P, P]),
        "kin_get_f": (c_int, [P, P]),
        "kin_sample_f": (c_int, [P, P, c_i64, P]),
        "kin_get_velocity": (c_int, [P, P]),
        "kin_step": (c_int, [P, c_int]),
        "kin_stats": (c_int, [P, P, P, P]),
        "kin_step_stats": (c_int, [P, c_int, P, P, P]),
        "kin_stats_async": (c_int, [P, P]),
        "kin_step_stats_async": (c_int, [P, c_int, P]),
        "kin_init_consistent": (c_int, [P, c_int, ctypes.c_double, P, P]),
        "kin_derived_stats": (c_int, [P, P, P]),
        "kin_num_shells": (c_int, [c_int]),
        "kin_sync": (c_int, [P]),
        "kin_step_launches": (c_int, [P]),
        "kin_set_tuning": (c_int, [P, c_int, c_int, c_int, c_int]),
        "kin_kernel_launches": (c_i64, [P]),
        "kin_get_nu": (c_double, [P]),
        "kin_get_dt": (c_double, [P]),
        "kin_get_time": (c_double, [P]),
        "kin_get_step": (c_i64, [P]),
        "kin_get_N": (c_int, [P]),
        "kin_get_scheme": (c_int, [P]),
        "kin_get_storage": (c_int, [P]),
        "kin_strerror": (ctypes.c_char_p, [c_int]),
        "kin_last_error": (ctypes.c_char_p, []),
        "kin_destroy": (None, [P]),
        "kin_energy_dissipation_noalloc": (c_int, [P, c_int, c_double, P, P]),
        "kin_check_guards": (c_int, [P]),
        "kin_test_corrupt_guard": (c_int, [P, c_int, c_int]),
        "kin_debug_status": (c_int, [P, P, c_int]),
        "kin_ensemble_create": (c_int, [P, c_int, P]),
        "kin_ensemble_set_tuning": (c_int, [P, c_int, c_int, c_int]),
        "kin_ensemble_step": (c_int, [P, c_int]),
        "kin_ensemble_test_timeout": (c_int, [P, c_double]),
        "kin_ensemble_info": (c_int, [P, P, P, P]),
        "kin_ensemble_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def load(build_if_needed: bool = True, debug: bool = False):
    """Load libkin.so, or with debug the index-checking build libkin_debug.so
    (building them with nvcc first if missing or stale).  A process loads one
    of the two: the first call decides."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _build

        path = DEBUG_LIB_PATH if debug else LIB_PATH
        if build_if_needed and not _build.up_to_date(path):
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError("%s not found; run paper_1601_03815_gb300.build" % path)
        _lib = _declare(ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL))
        return _lib


def debug_status(reset: bool = False):
    """kin_debug_status: (is_debug_build, first failed check or 0)."""
    isd = ctypes.c_int(0)
    word = ctypes.c_uint64(0)
    lib().kin_debug_status(ctypes.byref(isd), ctypes.byref(word), int(reset))
    return bool(isd.value), int(word.value)


def lib():
    return _lib if _lib is not None else load()


def _check(rc: int, where: str):
    if rc != KIN_OK:
        raise KinError(rc, where, lib().kin_last_error().decode())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def lattice():
    """D3Q19 velocities (19, 3) and weights (19,) in the library's order."""
    xi = np.zeros(57, dtype=np.int32)
    w = np.zeros(19, dtype=np.float64)
    _check(lib().kin_lattice(_ptr(xi), _ptr(w)), "kin_lattice")
    return xi.reshape(19, 3).astype(np.int64), w


def footprint_bytes(N: int, scheme: int, storage: int) -> int:
    return int(lib().kin_footprint_bytes(N, scheme, storage))


def num_shells(N: int) -> int:
    return int(lib().kin_num_shells(N))


def energy_dissipation_noalloc(u_ptr: int, N: int, nu: float, out_ptr: int, stream=None):
    """E and eps of a device velocity field u[3][N^3] (FP64) into the device
    array out[2], without any device allocation (see kin.h)."""
    _check(lib().kin_energy_dissipation_noalloc(ctypes.c_void_p(u_ptr), int(N), float(nu),
                                                 ctypes.c_void_p(out_ptr), _stream_handle(stream)),
           "kin_energy_dissipation_noalloc")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


class Sim:
    """One simulation (state resident in device memory)."""

    def __init__(self, N: int, scheme: int, nu: float, Ma: float = 0.1, dt: float | None = None,
                 storage: int = F32, stream=None):
        if dt is None:
            dt = 1.0 if scheme == LBE_MRT else 0.5
        h = ctypes.c_void_p()
        _check(lib().kin_create(int(N), int(scheme), float(nu), float(Ma), float(dt), int(storage),
                                _stream_handle(stream), ctypes.byref(h)), "kin_create")
        self._h = h
        self.N = int(N)
        self.scheme = int(scheme)
        self.storage = int(storage)

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().kin_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- state
    def init_field(self, seed: int, k0: float, re_lambda: float = 0.0):
        _check(lib().kin_init_field(self._h, ctypes.c_uint64(seed), float(k0), float(re_lambda)),
               "kin_init_field")

    def init_consistent(self, max_iter: int = 2000, tol: float = 0.0):
        """kin_init_consistent (MRT-LBE or DUGKS): iterate with the velocity
        held fixed until delta-rho changes by <= tol per iteration or max_iter
        iterations; returns (iterations, last measured change)."""
        it = ctypes.c_int(0)
        res = ctypes.c_double(0.0)
        _check(lib().kin_init_consistent(self._h, int(max_iter), float(tol), ctypes.byref(it), ctypes.byref(res)),
               "kin_init_consistent")
        return int(it.value), float(res.value)

    def set_velocity(self, u: np.ndarray):
        u = np.ascontiguousarray(u, dtype=np.float64)
        if u.shape != (3, self.N, self.N, self.N):
            raise ValueError("u must have shape (3, N, N, N)")
        _check(lib().kin_set_velocity(self._h, _ptr(u)), "kin_set_velocity")

    def set_f(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64)
        if f.shape != (19, self.N, self.N, self.N):
            raise ValueError("f must have shape (19, N, N, N)")
        _check(lib().kin_set_f(self._h, _ptr(f)), "kin_set_f")

    def get_f(self) -> np.ndarray:
        f = np.empty((19, self.N, self.N, self.N))
        _check(lib().kin_get_f(self._h, _ptr(f)), "kin_get_f")
        return f

    def sample_f(self, cells) -> np.ndarray:
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.empty((cells.size, 19))
        _check(lib().kin_sample_f(self._h, _ptr(cells), cells.size, _ptr(out)), "kin_sample_f")
        return out

    def get_velocity(self) -> np.ndarray:
        u = np.empty((3, self.N, self.N, self.N))
        _check(lib().kin_get_velocity(self._h, _ptr(u)), "kin_get_velocity")
        return u

    # -- time stepping and statistics
    def step(self, n: int = 1):
        _check(lib().kin_step(self._h, int(n)), "kin_step")

    def stats(self, spectrum: bool = False):
        """(E, eps) or (E, eps, Ek) of the current state."""
        E = np.zeros(1)
        eps = np.zeros(1)
        Ek = np.zeros(num_shells(self.N)) if spectrum else None
        _check(lib().kin_stats(self._h, _ptr(E), _ptr(eps), None if Ek is None else _ptr(Ek)),
               "kin_stats")
        if spectrum:
            return float(E[0]), float(eps[0]), Ek
        return float(E[0]), float(eps[0])

    def step_stats(self, n: int = 1, spectrum: bool = False):
        """kin_step_stats: n steps, then (E, eps) or (E, eps, Ek) of the new
        state; equal to step(n) followed by stats()."""
        E = np.zeros(1)
        eps = np.zeros(1)
        Ek = np.zeros(num_shells(self.N)) if spectrum else None
        _check(lib().kin_step_stats(self._h, int(n), _ptr(E), _ptr(eps), None if Ek is None else _ptr(Ek)),
               "kin_step_stats")
        if spectrum:
            return float(E[0]), float(eps[0]), Ek
        return float(E[0]), float(eps[0])

    def stats_async(self, out: np.ndarray):
        """kin_stats_async: enqueue (E, eps) of the current state into out[0:2]
        (float64, C-contiguous; page-locked memory, e.g. a pinned torch tensor's
        numpy view, keeps the call asynchronous) and return at once; the values
        are there once the stream has passed this point."""
        _check(lib().kin_stats_async(self._h, _out2(out)), "kin_stats_async")

    def step_stats_async(self, n: int, out: np.ndarray):
        """kin_step_stats_async: n steps, then stats_async(out) of the new state."""
        _check(lib().kin_step_stats_async(self._h, int(n), _out2(out)), "kin_step_stats_async")

    DERIVED = ("E", "uprime", "eps", "lambda", "Re_lambda", "eta", "S", "F")

    def derived_stats(self):
        """kin_derived_stats: dict of E, u', spectral eps, lambda, Re_lambda,
        eta, S, F and the dissipation spectrum D (per shell)."""
        out = np.zeros(8)
        D = np.zeros(num_shells(self.N))
        _check(lib().kin_derived_stats(self._h, _ptr(out), _ptr(D)), "kin_derived_stats")
        res = dict(zip(self.DERIVED, (float(v) for v in out)))
        res["D"] = D
        return res

    def set_tuning(self, block_x: int = 0, tile_y: int = 0, zchunk: int = 0, variant: int = -1):
        _check(lib().kin_set_tuning(self._h, int(block_x), int(tile_y), int(zchunk), int(variant)),
               "kin_set_tuning")

    @property
    def step_launches(self) -> int:
        return int(lib().kin_step_launches(self._h))

    @property
    def kernel_launches(self) -> int:
        return int(lib().kin_kernel_launches(self._h))

    def sync(self):
        _check(lib().kin_sync(self._h), "kin_sync")

    def check_guards(self):
        """kin_check_guards: raise KinError (KIN_EGUARD) if a guard region
        around a state buffer was overwritten."""
        _check(lib().kin_check_guards(self._h), "kin_check_guards")

    def corrupt_guard(self, buffer: int, side: int):
        """kin_test_corrupt_guard: change one byte of a guard region from the
        host, for tests of kin_check_guards."""
        _check(lib().kin_test_corrupt_guard(self._h, int(buffer), int(side)), "kin_test_corrupt_guard")

    @property
    def nu(self) -> float:
        return lib().kin_get_nu(self._h)

    @property
    def dt(self) -> float:
        return lib().kin_get_dt(self._h)

    @property
    def time(self) -> float:
        return lib().kin_get_time(self._h)

    @property
    def steps_taken(self) -> int:
        return int(lib().kin_get_step(self._h))


class Ensemble:
    """Independent simulations advanced together by one CUDA graph launch per
    step() call: a persistent kernel for the DUGKS members and, on a parallel
    stream, one batched launch per step for the LBE members (see
    kin_ensemble_* in kin.h).  Keeps references to its members so they
    outlive it."""

    def __init__(self, members):
        self.members = list(members)
        arr = (ctypes.c_void_p * len(self.members))(*[m.handle.value for m in self.members])
        h = ctypes.c_void_p()
        _check(lib().kin_ensemble_create(arr, len(self.members), ctypes.byref(h)), "kin_ensemble_create")
        self._h = h

    def set_tuning(self, tile_y: int = 0, zchunk: int = 0, lbe_block: int = 0):
        _check(lib().kin_ensemble_set_tuning(self._h, int(tile_y), int(zchunk), int(lbe_block)),
               "kin_ensemble_set_tuning")

    def step(self, n: int = 1):
        _check(lib().kin_ensemble_step(self._h, int(n)), "kin_ensemble_step")

    def test_timeout(self, seconds: float) -> int:
        """Run the bounded-wait self test; returns the status code."""
        return int(lib().kin_ensemble_test_timeout(self._h, float(seconds)))

    def info(self):
        nitems, grid, launches = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        _check(lib().kin_ensemble_info(self._h, ctypes.byref(nitems), ctypes.byref(grid),
                                       ctypes.byref(launches)), "kin_ensemble_info")
        return {"items": nitems.value, "grid": grid.value, "launches": launches.value}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().kin_ensemble_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
