"""bench.py's multi-rank host logic on CPU: world-size-2 gloo ranks check the
barrier and the max/sum reductions that turn per-rank times and unit counts into
the whole-job line (the GPU runs are replicas with no data-path collective)."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w, _ = bench.dist_setup(world)
    assert (r, w) == (rank, world)
    bench.barrier(w)
    ms = 10.0 + 5.0 * rank          # per-rank step time: the job is as slow as its slowest rank
    units = 1000.0 * (rank + 1)     # units each rank processed
    out[rank] = (bench.reduce_max(ms, w), bench.reduce_sum(units, w))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_rank_reductions():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (15.0, 3000.0)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5 and bench.reduce_sum(7.0, 1) == 7.0
    bench.barrier(1)
