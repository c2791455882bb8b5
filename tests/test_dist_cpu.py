"""The benchmark's multi-process path on CPU: two gloo ranks (torchrun-style
environment on 127.0.0.1) set up the group, meet at the barriers and agree on
the max-over-ranks time.  The path itself runs independent replicas, so these
helpers are its only cross-rank traffic."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    import torch.distributed as dist
    r, w = bench.dist_setup()
    assert (r, w) == (rank, world) and dist.get_backend() == "gloo"
    bench.dist_barrier(w)
    m = bench.dist_max(10.0 + 3.0 * rank, w)
    bench.dist_barrier(w)
    out[rank] = m
    dist.destroy_process_group()


def test_two_gloo_ranks_barrier_and_max_over_ranks():
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert dict(out) == {0: 13.0, 1: 13.0}
