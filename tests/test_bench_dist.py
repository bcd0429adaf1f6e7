"""Multi-rank bench logic on CPU: two gloo ranks, the whole-job value uses the
slowest rank's time and counts every rank's cell updates (weak scaling,
replicas with no collective on the data path)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = [1.5, 2.0][rank]
    tmax = bench.max_over_ranks(elapsed, dist, "cpu")
    value = bench.whole_job_mlups(2 * 256 ** 3, 100, world, tmax)
    w, r, l = bench._dist()
    out.put((rank, tmax, value, w, r, l))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, tmax, value, w, r, l in res:
        assert tmax == 2.0
        assert value == pytest.approx(2 * 2 * 256 ** 3 * 100 / 2.0 / 1e6)
        assert (w, r, l) == (2, rank, rank)


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.0, None) == 3.0
    cfg = bench.bench_config(256, "f32", 1)
    assert cfg["N"] == 256 and "256^3" in cfg["workload"] and cfg["parallelism"] == "single"
    assert "larger than L2" in cfg["l2"]
