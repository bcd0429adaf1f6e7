"""Domain decomposition of one periodic box over CPU ranks (gloo).

Each rank owns a slab of z planes.  Before every step it sends its bottom
plane to the rank below and its top plane to the rank above (periodic) and
receives one halo plane from each, steps the slab extended by the two halo
planes with the oracle, and keeps its own planes.  One halo plane per face is
all either scheme needs: an MRT-LBE cell receives populations only from its
face/edge neighbours, and the DUGKS update of a plane reads f-bar-plus one
plane away (the Eq. 19 pre-step is local, so the halo carries f-tilde).  The
gathered slabs must equal the single-box run bit for bit, because every
cell's arithmetic is the same wherever the cell sits.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NU = 0.017


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _bounds(nz, world):
    cuts = [round(r * nz / world) for r in range(world + 1)]
    return list(zip(cuts[:-1], cuts[1:]))


def _rank(rank, world, port, scheme, dt, f, steps, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist

    import oracle as orc

    orc.set_num_threads(1)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    z0, z1 = _bounds(f.shape[1], world)[rank]
    slab = np.ascontiguousarray(f[:, z0:z1])
    below, above = (rank - 1) % world, (rank + 1) % world
    for _ in range(steps):
        lo = torch.empty((19,) + slab.shape[2:], dtype=torch.float64)
        hi = torch.empty_like(lo)
        # tag 0: a bottom plane travelling down; tag 1: a top plane travelling up
        reqs = [
            dist.isend(torch.from_numpy(np.ascontiguousarray(slab[:, 0])), below, tag=0),
            dist.isend(torch.from_numpy(np.ascontiguousarray(slab[:, -1])), above, tag=1),
            dist.irecv(hi, above, tag=0),
            dist.irecv(lo, below, tag=1),
        ]
        for r in reqs:
            r.wait()
        ext = np.concatenate([lo.numpy()[:, None], slab, hi.numpy()[:, None]], axis=1)
        slab = orc.step(scheme, ext, NU, dt)[:, 1:-1].copy()
    out.put((rank, slab))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("scheme,dt", [("lbe", 1.0), ("dugks", 0.5)])
def test_two_rank_slab_decomposition_is_exact(orc, scheme, dt):
    rng = np.random.default_rng(77)
    nz, ny, nx = 7, 5, 6  # uneven slabs: 4 + 3 planes
    u = 0.05 * rng.standard_normal((3, nz, ny, nx))
    f = orc.equilibrium_field(u, 1e-2 * rng.standard_normal((nz, ny, nx)))
    f = f + 1e-3 * rng.standard_normal(f.shape)
    steps = 3
    ref = f
    for _ in range(steps):
        ref = orc.step(scheme, ref, NU, dt)

    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, scheme, dt, f, steps, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=180) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = np.concatenate([res[r] for r in range(world)], axis=1)
    np.testing.assert_array_equal(got, ref)
