"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/*.h declares (no GPU calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(kin_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ["kin_create", "kin_init_field", "kin_step", "kin_stats", "kin_destroy",
                     "kin_set_velocity", "kin_get_f", "kin_set_f"]:
        assert required in names


@pytest.fixture(scope="module")
def libkin():
    import paper_1601_03815_gb300 as kin

    return kin.load()


def test_library_exports_every_declared_symbol(libkin):
    missing = [n for n in _declared() if not hasattr(libkin, n)]
    assert not missing, missing


def test_library_is_built_for_sm103a():
    import paper_1601_03815_gb300.build as b

    assert "arch=compute_103a,code=sm_103a" in " ".join(b.ARCH)
    assert os.path.exists(b.LIB)


def test_host_only_entry_points(libkin):
    """Calls that touch no device: error strings, shell count, footprint,
    lattice order equal to the oracle's."""
    import numpy as np

    import paper_1601_03815_gb300 as kin

    assert libkin.kin_strerror(0) == b"ok"
    assert libkin.kin_strerror(-1) == b"invalid argument"
    assert kin.num_shells(32) == 1 + int(np.floor(np.sqrt(3 * 16 * 16) + 0.5))
    assert kin.footprint_bytes(256, kin.LBE_MRT, kin.F32) == 2 * 19 * 256 ** 3 * 4
    assert kin.footprint_bytes(256, kin.DUGKS, kin.F16) == 2 * 19 * 256 ** 3 * 2
    import oracle

    xi_o, w_o = oracle.lattice()
    xi_k, w_k = kin.lattice()
    np.testing.assert_array_equal(xi_k, xi_o)
    np.testing.assert_array_equal(w_k, w_o)


def test_invalid_arguments_are_rejected_without_a_device(libkin):
    """Argument validation happens before any CUDA call."""
    h = ctypes.c_void_p()
    assert libkin.kin_create(1, 0, 0.01, 0.1, 1.0, 0, None, ctypes.byref(h)) == -1
    assert libkin.kin_create(32, 7, 0.01, 0.1, 1.0, 0, None, ctypes.byref(h)) == -1
    assert libkin.kin_create(32, 0, -1.0, 0.1, 1.0, 0, None, ctypes.byref(h)) == -1
    assert libkin.kin_create(32, 0, 0.01, 0.1, 0.5, 0, None, ctypes.byref(h)) == -1  # LBE dt != 1
    assert libkin.kin_create(32, 1, 0.01, 0.1, 0.8, 0, None, ctypes.byref(h)) == -1  # DUGKS CFL > 1
    assert libkin.kin_create(32, 1, 0.01, 0.1, 0.5, 9, None, ctypes.byref(h)) == -1
    assert h.value is None
    assert b"DUGKS" in libkin.kin_last_error() or b"storage" in libkin.kin_last_error()
    # a NULL simulation is rejected by every entry point that takes one
    d = ctypes.c_double()
    assert libkin.kin_step(None, 1) == -1
    assert libkin.kin_step_stats(None, 1, ctypes.byref(d), ctypes.byref(d), None) == -1
    assert libkin.kin_init_consistent(None, 10, ctypes.c_double(0.0), None, None) == -1
    out = (ctypes.c_double * 2)()
    assert libkin.kin_stats_async(None, out) == -1
    assert libkin.kin_step_stats_async(None, 1, out) == -1
    libkin.kin_destroy(None)  # NULL-safe


def test_debug_library_exports_every_declared_symbol():
    """The KIN_DEBUG build (index checks in the stencil kernels) offers the
    same boundary."""
    import paper_1601_03815_gb300.build as b

    b.build()
    lib = ctypes.CDLL(b.DEBUG_LIB, mode=ctypes.RTLD_LOCAL)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
