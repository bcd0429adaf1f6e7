"""kin_step_stats: n steps and the statistics of the new state, bit for bit
equal to kin_step followed by kin_stats.

For DUGKS with FP32-computed storage the last fused step writes the velocity
of the state it produces and kin_stats skips its own velocity pass; these
tests check that the two routes agree exactly, that the cached velocity is
dropped whenever the state changes (set_f, steps, ensemble steps), and that
every other configuration takes the plain route.
"""
import numpy as np
import pytest

import kin_inputs as ki

pytestmark = pytest.mark.gpu


def _state(orc, N, seed):
    u = ki.dhit_velocity(N, seed, min(4.0, N / 4), 0.1)
    f = orc.equilibrium_field(u)
    return f + ki.random_populations(N, N, N, seed + 9, 2e-5)


def _pair(kin, scheme, N, storage, f0, variant=-1):
    dt = 1.0 if scheme == "lbe" else 0.5
    code = kin.LBE_MRT if scheme == "lbe" else kin.DUGKS
    sims = [kin.Sim(N, code, 0.011, 0.1, dt, storage) for _ in range(2)]
    for s in sims:
        if variant >= 0:
            s.set_tuning(0, 0, 0, variant)
        s.set_f(f0)
    return sims


@pytest.mark.parametrize("scheme", ["lbe", "dugks"])
@pytest.mark.parametrize("storage", [0, 1, 2, 3])
@pytest.mark.parametrize("N", [36, 64])
def test_step_stats_equals_step_then_stats(kin, orc, scheme, storage, N):
    a, b = _pair(kin, scheme, N, storage, _state(orc, N, 500 + N))
    ea = a.step_stats(3)
    b.step(3)
    eb = b.stats()
    assert ea == eb  # bitwise
    assert a.stats() == eb  # a second call reuses or recomputes the same velocity
    ka = a.step_stats(2, spectrum=True)
    b.step(2)
    kb = b.stats(spectrum=True)
    assert ka[:2] == kb[:2]
    np.testing.assert_array_equal(ka[2], kb[2])
    np.testing.assert_array_equal(a.get_f(), b.get_f())
    assert a.step_stats(0) == b.stats()
    a.close()
    b.close()


@pytest.mark.parametrize("variant", [1])
def test_step_stats_other_dugks_variants(kin, orc, variant):
    N = 36
    a, b = _pair(kin, "dugks", N, kin.F32, _state(orc, N, 61), variant)
    ea = a.step_stats(2)
    b.step(2)
    assert ea == b.stats()
    a.close()
    b.close()


def test_cached_velocity_follows_the_state(kin, orc):
    """After a fused step the velocity is cached; set_f, a plain step and an
    ensemble step each make kin_stats recompute it."""
    N = 32
    f0, f1 = _state(orc, N, 71), _state(orc, N, 72)
    a, b = _pair(kin, "dugks", N, kin.F32, f0)
    a.step_stats(1)
    # the fused velocity agrees with the FP64 velocity of the stored state
    u = a.get_velocity()
    E, _ = a.stats()
    assert abs(E / (0.5 * np.mean(np.sum(u * u, axis=0))) - 1) < 1e-6
    a.set_f(f1)
    b.set_f(f1)
    assert a.stats() == b.stats()
    a.step_stats(1)
    a.step(1)
    b.step(2)
    assert a.stats() == b.stats()
    a.step_stats(1)
    b.step(1)
    ens = kin.Ensemble([a])
    ens.step(2)
    ens.close()
    b.step(2)
    assert a.stats() == b.stats()
    a.close()
    b.close()


@pytest.mark.parametrize("scheme", ["lbe", "dugks"])
@pytest.mark.parametrize("storage", [0, 1, 3])
def test_async_statistics_equal_the_synchronous_ones(kin, orc, scheme, storage):
    """kin_stats_async and kin_step_stats_async deliver the kin_stats /
    kin_step_stats values bit for bit into page-locked host memory, also when
    a loop keeps several steps in flight and reads each result one step late
    (events recorded on the simulation's stream)."""
    import torch

    N, steps = 36, 6
    f0 = _state(orc, N, 700)
    dt = 1.0 if scheme == "lbe" else 0.5
    code = kin.LBE_MRT if scheme == "lbe" else kin.DUGKS
    stream = torch.cuda.Stream()
    a = kin.Sim(N, code, 0.011, 0.1, dt, storage, stream=stream)
    b = kin.Sim(N, code, 0.011, 0.1, dt, storage)
    a.set_f(f0)
    b.set_f(f0)
    out = torch.zeros((steps + 1, 2), dtype=torch.float64, pin_memory=True).numpy()
    a.stats_async(out[0])
    events = []
    for k in range(1, steps + 1):
        if k % 2:
            a.step_stats_async(1, out[k])
        else:
            a.step(1)
            a.stats_async(out[k])
        ev = torch.cuda.Event()
        ev.record(stream)
        events.append(ev)
        if k > 1:
            events[k - 2].synchronize()
            assert np.all(np.isfinite(out[k - 1]))
    a.sync()
    want = [b.stats()]
    for k in range(1, steps + 1):
        want.append(b.step_stats(1))
    np.testing.assert_array_equal(out, np.array(want))
    with pytest.raises(ValueError):
        a.stats_async(np.zeros(1))
    a.close()
    b.close()
