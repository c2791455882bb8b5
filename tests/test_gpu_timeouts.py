"""Every kind of bounded device wait, made to run out, reports GSP_ERR_TIMEOUT.

The library's waits are bounded and return an error status instead of
hanging: the grid barrier of the fused edge map, the depth sort's decoupled
look-back, and the waits for bulk / TMA copies
into shared memory (projection SH rows, edge-map halo boxes).  Each test
makes one kind of wait run out deterministically through the entry point's
failure-injection hook - a barrier that is never opened, a look-back word
that is never published, a copy wait that gives up at once (the block still
lets its own copies land before it leaves) - asserts that the call reports
exactly GSP_ERR_TIMEOUT, and then checks that a normal call on the same
context gives the same result as before the failure.  Nothing here faults,
traps or hangs a GPU: every wait that is made to run out has a short poll
limit, and no block leaves with a copy in flight.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

SHORT = 2000  # polls of a wait that is meant to run out


def _timeout(gsp):
    return gsp._lib.GSP_ERR_TIMEOUT


def _views(gsp, pitched, n=6):
    import torch
    imgs = [torch.from_numpy(synth.image(203, 347, 70 + i)).cuda() for i in range(n)]
    return [gsp.pitched_image(t, 16) for t in imgs] if pitched else imgs


@pytest.mark.parametrize("pitched,n", [(False, 6), (True, 6), (True, 64)])
def test_edge_grid_barrier_that_is_never_opened(gsp_lib, pitched, n):
    """Both fused schedules: 6 views (tile kernel) and 64 views of 203 x 347
    (4.5M pixels: walk kernel)."""
    import torch
    ts = _views(gsp_lib, pitched, n)
    E0, m0, _, s0 = gsp_lib.edge_map(ts)
    torch.cuda.synchronize()
    assert int(s0.item()) == 0
    _, _, _, st = gsp_lib.edge_map(ts, spin_limit=SHORT, test_expire=1)
    torch.cuda.synchronize()
    assert int(st.item()) == _timeout(gsp_lib)
    E1, m1, _, s1 = gsp_lib.edge_map(ts)
    torch.cuda.synchronize()
    assert int(s1.item()) == 0 and torch.equal(E0, E1) and torch.equal(m0, m1)


def test_edge_tma_box_wait_that_gives_up(gsp_lib):
    """Pitched (16-byte aligned) views of a small batch are staged by TMA; each
    block's wait for its box gives up at once, drains its copies and leaves."""
    import torch
    ts = _views(gsp_lib, True, n=32)
    E0, m0, _, s0 = gsp_lib.edge_map(ts)
    torch.cuda.synchronize()
    assert int(s0.item()) == 0
    _, _, _, st = gsp_lib.edge_map(ts, test_expire=2)
    torch.cuda.synchronize()
    assert int(st.item()) == _timeout(gsp_lib)
    E1, m1, _, s1 = gsp_lib.edge_map(ts)
    torch.cuda.synchronize()
    assert int(s1.item()) == 0 and torch.equal(E0, E1) and torch.equal(m0, m1)


def _render_scene(gsp, n=200_000, w=640, h=480):
    import torch
    g = synth.gaussians(n, 3, seed=11)
    cam = synth.camera_front(w, h)
    gs = gsp.GaussianSet.from_arrays(g)
    r = gsp.Renderer(gs, [cam], pair_capacity=1 << 25)
    out = r.forward()
    torch.cuda.synchronize()
    assert int(out["status"].item()) == 0
    return r, out


def test_depth_sort_lookback_that_never_completes(gsp_lib):
    """Tile 0 of the first sort pass withholds its digit counts: every later
    tile's look-back runs out, the pass raises the overflow flag and the
    forward pass skips the rest of its stages."""
    import torch
    r, ref = _render_scene(gsp_lib)
    rgb0, T0 = ref["rgb"].clone(), ref["T"].clone()
    r.spin_limit, r.test_expire = SHORT, 1
    out = r.forward()
    torch.cuda.synchronize()
    assert int(out["status"].item()) == _timeout(gsp_lib)
    r.spin_limit, r.test_expire = 0, 0
    again = r.forward()
    torch.cuda.synchronize()
    assert int(again["status"].item()) == 0
    assert torch.equal(again["rgb"], rgb0) and torch.equal(again["T"], T0)


def test_projection_copy_wait_that_gives_up(gsp_lib):
    """Each projection thread gives up on the bulk copy of its SH row at once
    and reads the row from global memory: the status says so, and the output
    is complete and identical."""
    import torch
    r, ref = _render_scene(gsp_lib)
    rgb0, T0, last0 = ref["rgb"].clone(), ref["T"].clone(), ref["last"].clone()
    r.test_expire = 2
    out = r.forward()
    torch.cuda.synchronize()
    assert int(out["status"].item()) == _timeout(gsp_lib)
    assert torch.equal(out["rgb"], rgb0) and torch.equal(out["T"], T0) and torch.equal(out["last"], last0)
    r.test_expire = 0
    again = r.forward()
    torch.cuda.synchronize()
    assert int(again["status"].item()) == 0 and torch.equal(again["rgb"], rgb0)
