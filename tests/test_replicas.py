"""The multi-GPU path of the benchmark runs independent replicas (a single
forest does not shard): each rank times its own instance and the whole-job
figures are the slowest rank's time and the sum of the ranks' cell updates.
This host logic is checked with two gloo ranks on the CPU."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    seconds = [2.0, 3.5][rank]
    units = [1000, 2500][rank]
    t, u = bench.combine_ranks(dist, seconds, units, "cpu")
    out[rank] = (t, u)
    dist.destroy_process_group()


def test_combine_ranks_two_gloo_ranks():
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (3.5, 3500.0)


def test_single_process_passes_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(None, 1.25, 77, "cpu") == (1.25, 77)
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK") if k in os.environ}
    try:
        assert bench.dist_setup() == (1, 0, 0)
    finally:
        os.environ.update(env)
