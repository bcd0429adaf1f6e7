"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (per population i, normalised by the oracle's max |f_i|, since f_i
is a deviation from W_i rho0 and is often near zero):
  FP64 storage  1e-12 after one step
  FP32 storage  1e-5 after one step (the stated target), measured ~1e-7
  FP16 storage  2e-3 (11-bit significand: half-ulp 4.9e-4 of max|f_i|)
  BF16 storage  1.6e-2 (8-bit significand: half-ulp 3.9e-3 of max|f_i|)
The one-step cases also report (test property) the pointwise relative error
with a floor, max |df_i| / max(|f_i|, 1e-3 W_i Ma), and hold it to the
tolerance above carried over to this measure: times max_i (max|f_i| / floor_i),
about 2000 here (|f_i| reaches ~0.2 W_i at Ma = 0.1).
"""
import numpy as np
import pytest

import kin_inputs as ki

pytestmark = pytest.mark.gpu

TOL = {3: 1e-12, 0: 1e-5, 1: 2e-3, 2: 1.6e-2}  # keyed by storage code


def _state(orc, N, seed, neq=True):
    """A turbulence-like FP64 state: DHIT velocity for even N, random
    velocity otherwise, plus a random non-equilibrium part."""
    if N % 2 == 0 and N >= 4:
        u = ki.dhit_velocity(N, seed, min(4.0, N / 4), 0.1)
    else:
        u = ki.random_velocity(N, N, N, seed, 0.03)
    drho = 1e-3 * np.random.default_rng(seed + 7).standard_normal((N, N, N))
    f = orc.equilibrium_field(u, drho)
    if neq:
        f = f + ki.random_populations(N, N, N, seed + 9, 2e-5)
    return f


def _err(got, ref):
    scale = np.abs(ref).reshape(19, -1).max(axis=1)
    return (np.abs(got - ref).reshape(19, -1).max(axis=1) / scale).max()


def _pointwise(orc, got, ref, Ma):
    """max |got - ref| / max(|ref|, 1e-3 W_i Ma) over all cells and i, and the
    factor max_i (max|ref_i| / floor_i) that converts a max-normalised bound."""
    _, w = orc.lattice()
    floor = 1e-3 * Ma * np.asarray(w)
    pw = float((np.abs(got - ref) / np.maximum(np.abs(ref), floor[:, None, None, None])).max())
    conv = float((np.abs(ref).reshape(19, -1).max(axis=1) / floor).max())
    return pw, conv


def _scheme(kin, name):
    return kin.LBE_MRT if name == "lbe" else kin.DUGKS


@pytest.mark.parametrize("scheme", ["lbe", "dugks", "dugks-split", "dugks-ty4"])
@pytest.mark.parametrize("storage", [3, 0, 1, 2])
@pytest.mark.parametrize("N", [2, 5, 12, 33, 36])
def test_one_step_parity(kin, orc, scheme, storage, N, record_property):
    nu, dt = 0.013, (1.0 if scheme == "lbe" else 0.5)
    f0 = _state(orc, N, 100 + N)
    sim = kin.Sim(N, _scheme(kin, scheme), nu, 0.1, dt, storage)
    if scheme == "dugks-split":
        sim.set_tuning(variant=1)
    elif scheme == "dugks-ty4":
        sim.set_tuning(tile_y=4, zchunk=3)
    scheme = scheme.split("-")[0]
    sim.set_f(f0)
    f_in = sim.get_f()  # the stored (rounded) state is what the GPU steps from
    if storage == 3:
        np.testing.assert_array_equal(f_in, f0)
    sim.step(1)
    got = sim.get_f()
    ref = orc.step(scheme, f0, nu, dt)
    assert _err(got, ref) < TOL[storage]
    pw, conv = _pointwise(orc, got, ref, 0.1)
    record_property("pointwise_with_floor", pw)
    assert pw < TOL[storage] * max(conv, 1.0), (pw, conv)
    sim.close()


@pytest.mark.parametrize("scheme", ["lbe", "dugks", "dugks-ty4", "dugks-zc"])
def test_one_step_parity_ragged_large(kin, orc, scheme):
    """Sizes spanning several thread blocks and z chunks with ragged tails
    (x tiles of 30 and 128, y tiles of 4 and 8, z chunks of 7, 11 and the
    default)."""
    N = 130 if scheme == "lbe" else (68 if scheme == "dugks-zc" else 67)
    nu, dt = 0.02, (1.0 if scheme == "lbe" else 0.35355)
    f0 = _state(orc, N, 5)
    sim = kin.Sim(N, _scheme(kin, scheme), nu, 0.1, dt, kin.F32)
    if scheme == "dugks-ty4":
        sim.set_tuning(tile_y=4, zchunk=7)
    elif scheme == "dugks-zc":
        sim.set_tuning(zchunk=11)
    scheme = scheme.split("-")[0]
    sim.set_f(f0)
    sim.step(1)
    assert _err(sim.get_f(), orc.step(scheme, f0, nu, dt)) < 1e-5
    sim.close()


@pytest.mark.parametrize("scheme", ["lbe", "dugks"])
def test_history_fp64_32cubed(kin, orc, scheme):
    """Config C1: 32^3, FP64 on both sides, 100 steps from the seeded field
    (k0 = 4, Ma = 0.1, nu from Re_lambda = 25); E(t), eps(t) every step and
    the final state agree to rounding."""
    N, steps = 32, 100
    u, info = ki.dhit_velocity(N, 1100, 4.0, 0.1, return_info=True)
    nu = ki.nu_from_re_lambda(info["u_prime"], info["omega"], 25.0)
    dt = 1.0 if scheme == "lbe" else 0.35355
    sim = kin.Sim(N, _scheme(kin, scheme), nu, 0.1, dt, kin.F64)
    sim.set_velocity(u)
    f = orc.equilibrium_field(u)
    for n in range(steps + 1):
        Eg, eg = sim.stats()
        Eo, eo = orc.stats(f, nu)
        assert abs(Eg / Eo - 1) < 1e-12 and abs(eg / eo - 1) < 1e-11, (n, Eg, Eo, eg, eo)
        if n < steps:
            sim.step(1)
            f = orc.step(scheme, f, nu, dt)
    assert _err(sim.get_f(), f) < 1e-11
    sim.close()


@pytest.mark.parametrize("scheme", ["lbe", "dugks"])
def test_history_fp32_32cubed(kin, orc, scheme):
    """FP32 storage, 100 steps: E(t) and eps(t) within 1e-4 relative of the
    FP64 oracle."""
    N, steps = 32, 100
    u, info = ki.dhit_velocity(N, 1100, 4.0, 0.1, return_info=True)
    nu = ki.nu_from_re_lambda(info["u_prime"], info["omega"], 25.0)
    dt = 1.0 if scheme == "lbe" else 0.35355
    sim = kin.Sim(N, _scheme(kin, scheme), nu, 0.1, dt, kin.F32)
    sim.set_velocity(u)
    f = orc.equilibrium_field(u)
    worst = 0.0
    for n in range(steps + 1):
        if n % 10 == 0:
            Eg, eg = sim.stats()
            Eo, eo = orc.stats(f, nu)
            worst = max(worst, abs(Eg / Eo - 1), abs(eg / eo - 1))
        if n < steps:
            sim.step(1)
            f = orc.step(scheme, f, nu, dt)
    assert worst < 1e-4, worst
    sim.close()


def test_init_field_matches_input_generator(kin, orc):
    """kin_init_field (device generator, cuFFT) reproduces the seeded field of
    kin_inputs and the viscosity for Re_lambda."""
    for N, k0, Ma, re in [(32, 4.0, 0.1, 25.0), (48, 8.0, 0.15, 70.0)]:
        u, info = ki.dhit_velocity(N, 77 + N, k0, Ma, return_info=True)
        nu = ki.nu_from_re_lambda(info["u_prime"], info["omega"], re)
        for scheme in (kin.LBE_MRT, kin.DUGKS):
            sim = kin.Sim(N, scheme, 1.0, Ma, 1.0 if scheme == kin.LBE_MRT else 0.5, kin.F64)
            sim.init_field(77 + N, k0, re)
            assert abs(sim.nu / nu - 1) < 1e-12
            ug = sim.get_velocity()
            assert np.abs(ug - u).max() < 1e-13 * np.abs(u).max()
            f = sim.get_f()
            np.testing.assert_allclose(f, orc.equilibrium_field(u), rtol=0, atol=1e-15)
            sim.close()


@pytest.mark.parametrize("storage", [3, 0, 1, 2])
def test_stats_match_oracle(kin, orc, storage):
    N = 24
    f0 = _state(orc, N, 3)
    sim = kin.Sim(N, kin.DUGKS, 0.02, 0.1, 0.5, storage)
    sim.set_f(f0)
    E, eps, Ek = sim.stats(spectrum=True)
    fin = sim.get_f()
    Eo, eo = orc.stats(fin, 0.02)
    _, uo = orc.macro(fin)
    Eko, _ = orc.spectrum(uo, kin.num_shells(N))
    # FP64 storage is summed in FP64 throughout; the FP32-computed storage
    # types form each cell's |u|^2 and s_ab s_ab in FP32 (a few roundings of
    # 6e-8 each) and sum them in FP64
    tol = 1e-12 if storage == 3 else 2e-6
    assert abs(E / Eo - 1) < tol and abs(eps / eo - 1) < tol, (E / Eo - 1, eps / eo - 1)
    # E(k): FP64 transforms for FP64 storage, FP32 transforms (FP64 shell sums)
    # otherwise
    if storage == 3:
        np.testing.assert_allclose(Ek, Eko, rtol=1e-10, atol=1e-14 * Eko.max())
    else:
        np.testing.assert_allclose(Ek, Eko, rtol=1e-5, atol=1e-8 * Eko.max())
    # fixed-order reductions: bitwise reproducible
    E2, eps2, Ek2 = sim.stats(spectrum=True)
    assert E2 == E and eps2 == eps and np.array_equal(Ek2, Ek)
    sim.close()


@pytest.mark.parametrize("scheme", ["lbe", "dugks"])
def test_sampled_parity_256(kin, orc, scheme):
    """Bench size 256^3 FP32, the launch configuration the benchmark times:
    one step from the seeded field; 64 sampled cells are recomputed by the
    oracle from their own 3^3 neighbourhood (which holds every input of a
    one-step update of the centre cell)."""
    N = 256
    u = ki.dhit_velocity(N, 1300, 8.0, 0.15)
    nu, dt = 0.0126, (1.0 if scheme == "lbe" else 0.5)
    sim = kin.Sim(N, _scheme(kin, scheme), nu, 0.15, dt, kin.F32)
    sim.set_velocity(u)
    sim.step(1)
    rng = np.random.default_rng(42)
    pts = rng.integers(0, N, size=(64, 3))
    pts[:4] = [[0, 0, 0], [N - 1, N - 1, N - 1], [0, N - 1, 5], [N - 1, 0, 0]]  # wrap corners
    cells = pts[:, 0] + N * (pts[:, 1] + N * pts[:, 2])
    got = sim.sample_f(cells)
    scale = np.zeros(19)
    errs = np.zeros((len(pts), 19))
    for k, (x, y, z) in enumerate(pts):
        idx = np.arange(-1, 2)
        patch = u[:, (z + idx)[:, None, None] % N, (y + idx)[None, :, None] % N,
                  (x + idx)[None, None, :] % N]
        fo = orc.step(scheme, orc.equilibrium_field(patch), nu, dt)[:, 1, 1, 1]
        errs[k] = np.abs(got[k] - fo)
        scale = np.maximum(scale, np.abs(fo))
    assert (errs.max(axis=0) / scale).max() < 1e-5
    sim.close()


@pytest.mark.parametrize("scheme", ["lbe", "dugks"])
def test_conservation_and_uniform_flow_at_256(kin, scheme):
    """Properties that hold at any size: a uniform flow is preserved and the
    total momentum of a turbulent field is conserved (FP32 rounding)."""
    N = 256
    dt = 1.0 if scheme == "lbe" else 0.5
    sim = kin.Sim(N, _scheme(kin, scheme), 0.0126, 0.15, dt, kin.F32)
    sim.set_velocity(ki.uniform_velocity(N, N, N, [0.02, -0.01, 0.03]))
    sim.step(3)
    u = sim.get_velocity()
    for c, v in enumerate([0.02, -0.01, 0.03]):
        assert np.abs(u[c] - v).max() < 1e-7
    sim.init_field(1400, 8.0, 70.0)
    p0 = sim.get_velocity().reshape(3, -1).sum(1)
    sim.step(5)
    p1 = sim.get_velocity().reshape(3, -1).sum(1)
    assert np.abs(p1 - p0).max() < 1e-8 * N ** 3  # mean drift below 1e-8 per cell
    sim.close()


def test_step_runs_on_a_torch_stream(kin, orc):
    import torch

    s = torch.cuda.Stream()
    N = 16
    f0 = _state(orc, N, 8)
    sim = kin.Sim(N, kin.LBE_MRT, 0.02, 0.1, 1.0, kin.F32, stream=s)
    sim.set_f(f0)
    sim.step(3)
    sim.sync()
    ref = f0
    for _ in range(3):
        ref = orc.lbe_step(ref, 0.02)
    assert _err(sim.get_f(), ref) < 1e-5
    sim.close()


def test_errors_and_edge_cases(kin):
    with pytest.raises(kin.KinError) as e:
        kin.Sim(32, kin.DUGKS, 0.01, 0.1, 0.9)
    assert e.value.code == kin.KIN_EINVAL
    sim = kin.Sim(7, kin.LBE_MRT, 0.01, 0.1, 1.0)
    with pytest.raises(kin.KinError):
        sim.init_field(1, 4.0, 25.0)  # odd N
    sim.step(0)
    assert sim.steps_taken == 0
    with pytest.raises(kin.KinError):
        sim.step(-1)
    with pytest.raises(kin.KinError):
        sim.sample_f([7 ** 3])
    E, eps = sim.stats()  # zero state
    assert E == 0.0 and eps == 0.0
    sim.close()


@pytest.mark.parametrize("case", [
    # DUGKS at CFL 0.9, the stability sweep's time step (Sec. IV.E): dt = 0.9 / sqrt(2)
    ("dugks", 0.9 / np.sqrt(2.0), 0.013),
    ("dugks", 0.9 / np.sqrt(2.0), 2e-7),
    # the sweep's smallest viscosities: tau = 3 nu = 6e-7 for DUGKS (c1 = 1 - c2
    # ~ 5e-6, b ~ 1.5), s9 -> 2 for MRT-LBE
    ("dugks", 0.5, 2e-7),
    ("lbe", 1.0, 5e-5),
    ("lbe", 1.0, 2e-7),
])
@pytest.mark.parametrize("storage", [3, 0])
@pytest.mark.parametrize("N", [12, 33])
def test_one_step_parity_sweep_regime(kin, orc, case, storage, N):
    """One step at the stability sweep's parameters (CFL 0.9 and viscosities
    down to 2e-7) against the oracle, at the tolerances of the plain regime."""
    scheme, dt, nu = case
    f0 = _state(orc, N, 700 + N)
    sim = kin.Sim(N, _scheme(kin, scheme), nu, 0.1, dt, storage)
    sim.set_f(f0)
    f_in = sim.get_f()
    sim.step(1)
    got = sim.get_f()
    ref = orc.step(scheme, f_in, nu, dt)
    assert _err(got, ref) < TOL[storage]
    sim.close()


@pytest.mark.parametrize("storage", [0, 1, 2])
def test_lbe_block_sizes_above_the_launch_bounds(kin, storage):
    """block_x beyond the LBE kernels' 256 threads is clamped, not a failed
    launch: N = 264 (FP32: one cell a thread; FP16/BF16: four cells, N % 4 == 0)
    and N = 262 (two cells) give the default block's results bit for bit."""
    import kin_inputs as ki

    for N in (264, 262) if storage else (264,):
        u = ki.random_velocity(N, N, N, 41, 0.03)
        ref = kin.Sim(N, kin.LBE_MRT, 0.02, 0.1, 1.0, storage)
        ref.set_velocity(u)
        ref.step(2)
        want = ref.sample_f(list(range(0, N ** 3, 9973)))
        ref.close()
        for bx in (512, 1024):
            sim = kin.Sim(N, kin.LBE_MRT, 0.02, 0.1, 1.0, storage)
            sim.set_tuning(block_x=bx)
            sim.set_velocity(u)
            sim.step(2)
            np.testing.assert_array_equal(sim.sample_f(list(range(0, N ** 3, 9973))), want)
            sim.close()


@pytest.mark.parametrize("storage", [0, 1, 3])
def test_fused_dugks_results_do_not_depend_on_the_tile_shape(kin, orc, storage):
    """The fused DUGKS step gives the same bits for every tile height and z
    chunk (a cell's arithmetic does not depend on which tile or plane range
    computes it); N = 38 makes every shape ragged."""
    N = 38
    f0 = _state(orc, N, 4242)
    outs = []
    for ty, zc in ((8, 0), (4, 3), (8, 7), (4, 38)):
        if storage == 3 and ty == 8:
            continue  # FP64 storage always runs 4-row tiles
        sim = kin.Sim(N, kin.DUGKS, 0.013, 0.1, 0.5, storage)
        sim.set_tuning(tile_y=ty, zchunk=zc if zc else 0)
        sim.set_f(f0)
        sim.step(3)
        outs.append(sim.get_f())
        sim.close()
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])
