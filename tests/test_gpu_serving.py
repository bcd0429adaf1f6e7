"""Serving on the GPU with both backends (per-simulation streams, persistent
ensemble kernel): each request's final state is bitwise the same alone and
in the mix, and later arrivals join running requests."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _requests():
    from paper_1601_03815_gb300.serving import Request

    return [Request(rid=0, N=16, scheme=0, re_lambda=25.0, steps=37, seed=11, arrival=0.0, want_f=True),
            Request(rid=1, N=20, scheme=1, re_lambda=30.0, steps=52, seed=12, arrival=0.0, want_f=True),
            Request(rid=2, N=12, scheme=1, re_lambda=22.0, steps=19, seed=13, arrival=0.0, want_f=True),
            Request(rid=3, N=24, scheme=0, re_lambda=40.0, steps=44, seed=14, arrival=0.0, want_f=True)]


@pytest.mark.parametrize("backend", ["streams", "ensemble"])
def test_result_is_the_same_alone_and_in_the_mix(kin, backend):
    from paper_1601_03815_gb300.serving import BACKENDS, Server

    GpuBackend = BACKENDS[backend]
    reqs = _requests()
    be = GpuBackend()
    mix, rep = Server(be, hbm_budget=2 ** 31, max_active=8, chunk=10).run(reqs)
    be.close()
    assert rep["completed"] == len(reqs) and rep["max_active"] == len(reqs)
    for r in reqs:
        be1 = GpuBackend()
        alone, _ = Server(be1, hbm_budget=2 ** 31, max_active=1, chunk=7).run([r])
        be1.close()
        m = [x for x in mix if x.rid == r.rid][0]
        np.testing.assert_array_equal(alone[0].f, m.f)
        assert alone[0].E == m.E and alone[0].eps == m.eps


@pytest.mark.parametrize("backend", ["streams", "ensemble"])
def test_requests_arriving_later_join_running_ones(kin, backend):
    from paper_1601_03815_gb300.serving import BACKENDS, Request, Server

    GpuBackend = BACKENDS[backend]
    # the first request runs long enough (1000 ticks) that the later arrivals
    # find it still resident however fast a tick is
    reqs = [Request(rid=k, N=16, scheme=k % 2, re_lambda=25.0, steps=20000 if k == 0 else 400,
                    seed=20 + k, arrival=0.01 * k) for k in range(5)]
    be = GpuBackend()
    res, rep = Server(be, hbm_budget=2 ** 31, max_active=8, chunk=20).run(reqs)
    be.close()
    assert rep["completed"] == 5 and rep["max_active"] >= 2
    assert all(np.isfinite(r.E) and r.E > 0 for r in res)
