"""The N > 1 path of bench.py on CPU: world-size-2 gloo ranks, each running an
independent replica.  The whole-job step time is the slowest rank's and the particle
count is every rank's (weak scaling; no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, q):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [10.0, 25.0][rank]
    n_local = [1000, 3000][rank]
    ms, value = bench.across_ranks(ms_local, n_local, dist, "cpu")
    dist.barrier()
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_rank_weak_scaling_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for _, ms, value in res:
        assert ms == 25.0
        assert value == pytest.approx(4000 / 25e-3)


def test_single_rank_is_identity():
    import bench
    ms, value = bench.across_ranks(20.0, 1000)
    assert ms == 20.0 and value == pytest.approx(1000 / 20e-3)
