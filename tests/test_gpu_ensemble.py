"""Ensembles (persistent DUGKS kernel beside batched LBE launches, one graph):
each member is bitwise identical to stepping it alone with kin_step and
whether it runs alone in an ensemble or mixed with other members, across odd
and even step counts, graph re-launches, graphs split at 256 steps, ragged
tiles and FP32/FP16/BF16 storage; members match the FP64 oracle; the member
barrier is bounded and reports KIN_ETIMEOUT, after which members refuse work
until set."""
import numpy as np
import pytest

import kin_inputs as ki

pytestmark = pytest.mark.gpu

MEMBERS = [("lbe", 16), ("dugks", 16), ("lbe", 20), ("dugks", 33), ("dugks", 12), ("lbe", 9)]


def _state(orc, N, seed):
    u = ki.random_velocity(N, N, N, seed, 0.03)
    return orc.equilibrium_field(u) + ki.random_populations(N, N, N, seed + 1, 1e-5)


def _make(kin, orc, tuning=(8, 16)):
    ens_members, solo = [], []
    for k, (scheme, N) in enumerate(MEMBERS):
        f0 = _state(orc, N, 300 + k)
        sc = kin.LBE_MRT if scheme == "lbe" else kin.DUGKS
        dt = 1.0 if scheme == "lbe" else 0.45
        nu = 0.01 + 0.002 * k
        a = kin.Sim(N, sc, nu, 0.1, dt, kin.F32)
        b = kin.Sim(N, sc, nu, 0.1, dt, kin.F32)
        a.set_f(f0)
        b.set_f(f0)
        b.set_tuning(tile_y=tuning[0], zchunk=tuning[1])
        ens_members.append(a)
        solo.append(b)
    return ens_members, solo


@pytest.mark.parametrize("tuning", [(8, 16), (4, 7), (6, 16)])
def test_ensemble_is_bitwise_equal_to_solo_runs(kin, orc, tuning):
    # a solo run has no 6-row tiles; a cell's arithmetic does not depend on the tile
    members, solo = _make(kin, orc, (8, 16) if tuning[0] == 6 else tuning)
    ens = kin.Ensemble(members)
    ens.set_tuning(tile_y=tuning[0], zchunk=tuning[1], lbe_block=128)
    ens.step(3)
    ens.step(4)  # second launch, other parity
    ens.step(3)  # graph for 3 steps reused
    for s in solo:
        s.step(10)
    for a, b in zip(members, solo):
        assert a.steps_taken == 10
        np.testing.assert_array_equal(a.get_f(), b.get_f())
    info = ens.info()
    assert info["launches"] == 3 and info["grid"] >= 1 and info["items"] > len(MEMBERS)
    ens.close()
    for s in members + solo:
        s.close()


def test_ensemble_members_match_the_oracle(kin, orc):
    """Each member of a mixed ensemble (both schemes, uneven N, ragged tiles,
    two launches) against the FP64 oracle stepped alone, element by element:
    max |f_i - f_i^oracle| / max |f_i^oracle| <= 1e-5 per population."""
    members, states = [], []
    specs = [("lbe", 8, 0.011), ("dugks", 12, 0.013), ("dugks", 9, 0.02), ("lbe", 13, 0.017),
             ("dugks", 16, 0.009)]
    for k, (scheme, N, nu) in enumerate(specs):
        f0 = _state(orc, N, 900 + k)
        dt = 1.0 if scheme == "lbe" else 0.45
        sim = kin.Sim(N, kin.LBE_MRT if scheme == "lbe" else kin.DUGKS, nu, 0.1, dt, kin.F32)
        sim.set_f(f0)
        members.append((sim, scheme, nu, dt))
        states.append(sim.get_f())  # the stored FP32 state the GPU steps from
    ens = kin.Ensemble([m[0] for m in members])
    ens.set_tuning(tile_y=4, zchunk=5, lbe_block=128)
    ens.step(2)
    ens.step(1)
    for (sim, scheme, nu, dt), f in zip(members, states):
        ref = f
        for _ in range(3):
            ref = orc.step(scheme, ref, nu, dt)
        got = sim.get_f()
        scale = np.abs(ref).reshape(19, -1).max(axis=1)
        err = (np.abs(got - ref).reshape(19, -1).max(axis=1) / scale).max()
        assert err < 1e-5, (scheme, sim.N, err)
        sim.close()
    ens.close()


def test_ensemble_barrier_timeout_is_bounded_and_harmless(kin, orc):
    import time

    members, solo = _make(kin, orc)
    ens = kin.Ensemble(members)
    before = [m.get_f() for m in members]
    t0 = time.time()
    rc = ens.test_timeout(0.05)
    assert rc == kin.KIN_ETIMEOUT
    assert time.time() - t0 < 30.0
    for m, f in zip(members, before):
        assert m.steps_taken == 0
        # the stall was at step 1 of 2, so the state is in fact untouched ...
        np.testing.assert_array_equal(m.get_f(), f)
        # ... but a timed-out launch leaves every member refusing work until set
        with pytest.raises(kin.KinError) as e:
            m.step(1)
        assert e.value.code == kin.KIN_ESTATE
    with pytest.raises(kin.KinError) as e:
        ens.step(1)
    assert e.value.code == kin.KIN_ESTATE
    for m, f in zip(members, before):
        m.set_f(f)
    # the ensemble works again afterwards
    ens.step(2)
    for s in solo:
        s.step(2)
    for a, b in zip(members, solo):
        fa, fb = a.get_f(), b.get_f()
        assert np.abs(fa - fb).max() < 1e-5 * np.abs(fb).max()
    ens.close()


def test_member_alone_and_in_the_mix_are_bitwise_equal(kin, orc):
    """The same member stepped by an ensemble of one and by the full ensemble
    gives identical bits: the mix changes the schedule, not the arithmetic."""
    members, _ = _make(kin, orc)
    alone = []
    for k, m in enumerate(members):
        c = kin.Sim(m.N, m.scheme, 0.01 + 0.002 * k, 0.1, 1.0 if m.scheme == kin.LBE_MRT else 0.45,
                    kin.F32)
        c.set_f(m.get_f())
        alone.append(c)
    mix = kin.Ensemble(members)
    mix.step(5)
    for c in alone:
        e1 = kin.Ensemble([c])
        e1.step(5)
        e1.close()
    for a, c in zip(members, alone):
        np.testing.assert_array_equal(a.get_f(), c.get_f())
    mix.close()


@pytest.mark.parametrize("tile_y", [6, 8])
def test_mixed_storage_members_are_bitwise_equal_to_solo_runs(kin, orc, tile_y):
    """FP16 and BF16 members (LBE at N % 4 == 0, N % 4 == 2 and odd N; DUGKS at
    even N) beside FP32 ones: bitwise the solo kin_step result, with 6-row
    tiles (the default beside LBE members) and 8-row ones."""
    specs = [("lbe", 16, kin.F16), ("lbe", 18, kin.BF16), ("lbe", 9, kin.F16), ("dugks", 16, kin.F16),
             ("dugks", 14, kin.BF16), ("dugks", 12, kin.F32), ("lbe", 12, kin.F32)]
    members, solo = [], []
    for k, (scheme, N, st) in enumerate(specs):
        f0 = _state(orc, N, 500 + k)
        sc = kin.LBE_MRT if scheme == "lbe" else kin.DUGKS
        dt = 1.0 if scheme == "lbe" else 0.45
        a = kin.Sim(N, sc, 0.012 + 0.001 * k, 0.1, dt, st)
        b = kin.Sim(N, sc, 0.012 + 0.001 * k, 0.1, dt, st)
        a.set_f(f0)
        b.set_f(f0)
        b.set_tuning(tile_y=8, zchunk=5)
        members.append(a)
        solo.append(b)
    ens = kin.Ensemble(members)
    ens.set_tuning(tile_y=tile_y, zchunk=5)
    ens.step(2)
    ens.step(3)
    for s in solo:
        s.step(5)
    for a, b in zip(members, solo):
        np.testing.assert_array_equal(a.get_f(), b.get_f())
    ens.close()
    for s in members + solo:
        s.close()


@pytest.mark.parametrize("schemes", ["lbe", "dugks"])
def test_single_scheme_ensembles_and_long_calls(kin, orc, schemes):
    """An ensemble of one scheme (no fork in the graph; an LBE-only one has no
    persistent launch) and a call of 300 steps (two graphs when there are LBE
    members) give the solo results bitwise."""
    Ns = (10, 16, 7)
    members, solo = [], []
    for k, N in enumerate(Ns):
        f0 = _state(orc, N, 700 + k)
        sc = kin.LBE_MRT if schemes == "lbe" else kin.DUGKS
        dt = 1.0 if schemes == "lbe" else 0.45
        a = kin.Sim(N, sc, 0.02, 0.1, dt, kin.F32)
        b = kin.Sim(N, sc, 0.02, 0.1, dt, kin.F32)
        a.set_f(f0)
        b.set_f(f0)
        members.append(a)
        solo.append(b)
    ens = kin.Ensemble(members)
    steps = 300
    ens.step(steps)
    for s in solo:
        s.set_tuning(tile_y=8, zchunk=16)
        s.step(steps)
    for a, b in zip(members, solo):
        assert a.steps_taken == steps
        np.testing.assert_array_equal(a.get_f(), b.get_f())
    info = ens.info()
    assert info["launches"] == (2 if schemes == "lbe" else 1)
    assert (info["grid"] == 0) == (schemes == "lbe")
    if schemes == "lbe":
        assert ens.test_timeout(0.05) == kin.KIN_EINVAL
    ens.close()
    for s in members + solo:
        s.close()


def test_ensemble_rejects_bad_members(kin):
    a = kin.Sim(8, kin.LBE_MRT, 0.01, 0.1, 1.0, kin.F64)
    with pytest.raises(kin.KinError):
        kin.Ensemble([a])
    b = kin.Sim(8, kin.LBE_MRT, 0.01, 0.1, 1.0, kin.F32)
    with pytest.raises(kin.KinError):
        kin.Ensemble([b, b])
    c = kin.Sim(9, kin.DUGKS, 0.01, 0.1, 0.5, kin.F16)  # 2-byte DUGKS needs an even N
    with pytest.raises(kin.KinError):
        kin.Ensemble([b, c])
    ens = kin.Ensemble([b])
    with pytest.raises(kin.KinError):
        ens.set_tuning(lbe_block=256)
    ens.close()
    for s in (a, b, c):
        s.close()
