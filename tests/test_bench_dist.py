"""The multi-rank path of bench.py on CPU: two gloo ranks reduce their step
times to the maximum and report whole-job DOF/s (replicas, weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    os.environ["CUDA_VISIBLE_DEVICES"] = ""
    import bench
    r, w, local, red_max, barrier = bench._dist()
    barrier()
    ms = red_max(10.0 + 5.0 * r)              # rank 1 is the slower one
    out[r] = (r, w, ms, bench.aggregate(1000.0, ms, w))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        rank, w, ms, value = out[r]
        assert w == world and ms == 15.0
        assert abs(value - 2 * 1000.0 / 0.015) < 1e-6
