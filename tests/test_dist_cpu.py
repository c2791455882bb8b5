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


# ---- view-sharded data parallelism (host logic): partition, flat buffer, all-reduce

def test_partition_views_is_balanced_deterministic_and_complete():
    from paper_2603_08661_gb300.sharded import partition_views
    import synth
    px = [w * h for (w, h) in synth.RING_RESOLUTIONS]
    for world in (1, 2, 3, 4, 8, 11):
        parts = partition_views(px, world)
        assert len(parts) == world
        flat = sorted(v for p in parts for v in p)
        assert flat == list(range(len(px)))  # every view exactly once
        assert parts == partition_views(px, world)
        loads = [sum(px[v] for v in p) for p in parts]
        if world <= len(px):
            # greedy largest-first: no rank exceeds the lightest by more than the largest view
            assert max(loads) - min(loads) <= max(px)
            assert all(p for p in parts)
        else:
            assert sum(1 for p in parts if not p) == world - len(px)
    assert partition_views([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]  # ties: lower index first, lower rank first


def test_flat_grads_views_tile_the_buffer():
    import torch
    from paper_2603_08661_gb300.sharded import FlatGrads
    f = FlatGrads(7, 3, device="cpu")
    assert f["means"].shape == (7, 3) and f["quats"].shape == (7, 4) and f["sh"].shape == (7, 16, 3)
    assert f["opacity_logits"].shape == (7,) and f["score"].shape == (7,) and f["loss"].shape == (1,)
    assert f.flat.numel() == 7 * (3 + 3 + 4 + 1 + 48 + 1) + 1
    for i, name in enumerate(("means", "log_scales", "quats", "opacity_logits", "sh", "score", "loss")):
        f[name].fill_(float(i + 1))
    # the views partition the buffer: every element written exactly once
    counts = torch.bincount(f.flat.long(), minlength=8)
    assert counts[0] == 0 and counts[1:].sum() == f.flat.numel()


def _sharded_rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    from paper_2603_08661_gb300.sharded import FlatGrads, all_reduce_flat, partition_views
    import synth
    px = [w * h for (w, h) in synth.RING_RESOLUTIONS]
    mine = partition_views(px, world)[rank]
    f = FlatGrads(50, 3, device="cpu")
    # stand-in for each rank's renders: every view adds a view-specific pattern
    for v in mine:
        g = torch.Generator().manual_seed(1000 + v)
        f.flat.add_(torch.randn(f.flat.numel(), generator=g))
    all_reduce_flat(f.flat)
    out[rank] = f.flat.numpy().copy()
    dist.destroy_process_group()


def test_two_gloo_ranks_all_reduce_equals_the_sum_over_all_views():
    import numpy as np
    import torch
    port = _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    procs = [ctx.Process(target=_sharded_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    n = 50 * (3 + 3 + 4 + 1 + 48 + 1) + 1
    ref = np.zeros(n, np.float64)
    for v in range(8):
        g = torch.Generator().manual_seed(1000 + v)
        ref += torch.randn(n, generator=g).double().numpy()
    assert np.array_equal(out[0], out[1])  # every rank holds the same sums
    np.testing.assert_allclose(out[0], ref, rtol=1e-5, atol=1e-5)
