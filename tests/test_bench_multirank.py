"""Host logic of the multi-process bench path on CPU (gloo, two ranks): the timing maximum over
ranks, the whole-job throughput and the per-rank workloads."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r "took" 1 + r seconds of steps and 10 - r seconds end to end
        mx = bench.max_over_ranks([1.0 + rank, 10.0 - rank], "cpu")
        wl = bench.make_workload("small", bench.rank_seed(0, rank))[0]
        out[rank] = (mx, float(wl.poses[0][4]), float(wl.poses[0][5]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_reduce_max_and_draw_distinct_gels():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == [2.0, 10.0]
    assert (res[0][1], res[0][2]) != (res[1][1], res[1][2])  # different seeded indenter offsets
    sys.path.insert(0, ROOT)
    import bench
    # whole-job throughput: all ranks' gel steps over the slowest rank's time
    assert bench.job_throughput(2, 1, 10, 2.0) == 10.0
