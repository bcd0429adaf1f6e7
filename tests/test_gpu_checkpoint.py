"""Checkpoint / resume through the canonical host layout: n steps in one go
equal n/2 steps, kin_get_f -> kin_set_f into a fresh simulation, n/2 steps,
bit for bit (the FP64 host copy holds every storage type exactly)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("scheme", ["lbe", "dugks"])
@pytest.mark.parametrize("storage", [0, 1, 2, 3])
def test_resume_is_bitwise(kin, scheme, storage):
    N, n = 20, 12
    sc = kin.LBE_MRT if scheme == "lbe" else kin.DUGKS
    dt = 1.0 if scheme == "lbe" else 0.5
    a = kin.Sim(N, sc, 0.02, 0.1, dt, storage)
    a.init_field(99, 4.0, 0.0)
    b = kin.Sim(N, sc, 0.02, 0.1, dt, storage)
    b.set_f(a.get_f())
    a.step(n)
    b.step(n // 2)
    snap = b.get_f()
    c = kin.Sim(N, sc, 0.02, 0.1, dt, storage)
    c.set_f(snap)
    c.step(n - n // 2)
    np.testing.assert_array_equal(a.get_f(), c.get_f())
    for s in (a, b, c):
        s.close()
