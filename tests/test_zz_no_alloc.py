"""The allocation-free E / eps entry point gives the same result as kin_stats.

kin_energy_dissipation_noalloc serves callers that cannot let the library
allocate device memory (a real-time loop that must not call cudaMalloc or
cudaFree, which can synchronise the device; an application whose device
memory belongs to its own allocator).  Its scratch is a fixed array inside the
library, so two calls in a row must both be right: the second reuses what the
first left there.  This file is collected last so that a run stopping at the
first failure has run every other test before it.
"""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_energy_dissipation_matches_kin_stats(kin):
    import torch

    N, nu = 24, 0.02
    # FP64 storage: kin_stats then sums in FP64 exactly as the no-alloc path does
    sim = kin.Sim(N, kin.LBE_MRT, nu, 0.1, 1.0, kin.F64)
    sim.init_field(11, 4.0, 0.0)
    E_ref, eps_ref = sim.stats()
    u = torch.from_numpy(sim.get_velocity()).cuda().contiguous()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(2):
        out.fill_(-1.0)
        kin.energy_dissipation_noalloc(u.data_ptr(), N, nu, out.data_ptr(), stream)
        torch.cuda.synchronize()
        E, eps = out.tolist()
        assert abs(E / E_ref - 1) < 1e-12 and abs(eps / eps_ref - 1) < 1e-12, (E, E_ref, eps, eps_ref)
    # a second field through the same fixed scratch
    sim.init_field(12, 4.0, 0.0)
    E2_ref, eps2_ref = sim.stats()
    u2 = torch.from_numpy(sim.get_velocity()).cuda().contiguous()
    kin.energy_dissipation_noalloc(u2.data_ptr(), N, nu, out.data_ptr(), stream)
    torch.cuda.synchronize()
    E2, eps2 = out.tolist()
    assert abs(E2 / E2_ref - 1) < 1e-12 and abs(eps2 / eps2_ref - 1) < 1e-12
    sim.close()


def test_noalloc_fills_every_partial_slot_against_the_oracle(kin, orc):
    """N = 144 needs more blocks than the fixed array holds partials for, so
    the reduction runs with every one of its slots; E and eps against the FP64
    oracle's definitions of the same field, on two calls in a row."""
    import numpy as np
    import torch

    import kin_inputs as ki

    N, nu = 144, 0.015
    u_h = ki.dhit_velocity(N, 21, 8.0, 0.1)
    E_o, eps_o = orc.energy_dissipation(u_h, nu)
    u = torch.from_numpy(np.ascontiguousarray(u_h)).cuda()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(-1.0)
        kin.energy_dissipation_noalloc(u.data_ptr(), N, nu, out.data_ptr(), torch.cuda.current_stream())
        torch.cuda.synchronize()
        E, eps = out.tolist()
        assert abs(E / E_o - 1) < 1e-12 and abs(eps / eps_o - 1) < 1e-12, (E, E_o, eps, eps_o)


def test_noalloc_rejects_sizes_beyond_its_scratch(kin):
    lib = kin.lib()
    rc = lib.kin_energy_dissipation_noalloc(ctypes.c_void_p(16), 2048, 0.01, ctypes.c_void_p(16), None)
    assert rc == kin.KIN_EINVAL
    assert b"1024" in lib.kin_last_error()
    rc = lib.kin_energy_dissipation_noalloc(None, 32, 0.01, None, None)
    assert rc == kin.KIN_EINVAL
