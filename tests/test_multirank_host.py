"""The N > 1 harness on CPU: replicas rendezvous over gloo (127.0.0.1), the
step time is the maximum over ranks and the throughput counts every rank's
units (weak scaling, no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    w, r, local = bench.dist_setup("gloo")
    t = bench.max_over_ranks(1.5 + r, w)              # rank times 1.5 s, 2.5 s
    v = bench.job_throughput(1024, 10, w, t)
    q.put((r, w, local, t, v))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, w, local, t, v) in enumerate(out):
        assert (rank, w, local) == (r, world, r)
        assert t == 2.5
        assert v == pytest.approx(1024 * 10 * 2 / 2.5)


def test_single_rank_is_a_no_op():
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.job_throughput(100, 4, 1, 2.0) == 200.0
