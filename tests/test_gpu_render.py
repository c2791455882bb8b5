"""GPU splatting parity against the FP64 oracle, through the C ABI.

Tolerances: rendered RGB and T_final within 1e-4 absolute; per-Gaussian edge
scores within 1e-4 relative; every gradient entry within 1e-4 relative of the
oracle's analytic adjoint (floor 1e-3 x the RMS of the parameter group) plus
the FP32 rounding bound 64 u A of entries whose terms cancel
(conftest.grad_bound), and within 1e-3 relative of central finite differences
(floor 1e-3 x RMS).  Pixels whose oracle evaluation meets a gate (alpha =
1/255, T (1 - alpha) = 1e-4) within GATE_REL relative are exempt, and so are
the Gaussians composited at such pixels, for the score and gradient checks;
their count must stay within EXEMPT_FRAC of the pixels compared.
"""
import math

import numpy as np
import pytest

import synth
from conftest import EXEMPT_FRAC, GATE_REL, assert_grads_match
from oracle import edge as oe
from oracle import raster as orc
from oracle import densify as od

pytestmark = pytest.mark.gpu

GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _flat_edge(edges):
    return np.concatenate([e.ravel() for e in edges]).astype(np.float32)


def gpu_render(gsp, g, cams, targets=None, edges=None, dL=None, pair_capacity=1 << 22, score_in="fwd",
               capacity=None, list_prefix=0):
    import torch
    dev = torch.device("cuda")
    gs = gsp.GaussianSet.from_arrays(g, capacity=capacity, device=dev)
    r = gsp.Renderer(gs, cams, pair_capacity, device=dev)
    r.list_prefix = list_prefix
    E = torch.from_numpy(_flat_edge(edges)).to(dev) if edges is not None else None
    score = torch.zeros(gs.capacity, device=dev) if E is not None else None
    tg = [torch.from_numpy(t).to(dev) for t in targets] if targets is not None else None
    out = r.forward(targets=tg, edge=E, score=score if score_in == "fwd" else None)
    grads = None
    if dL is not None or tg is not None:
        dl = torch.from_numpy(np.ascontiguousarray(dL, dtype=np.float32)).to(dev) if dL is not None else None
        grads = r.backward(out, targets=tg if dl is None else None, dL_drgb=dl, edge=E,
                           score=score if score_in == "bwd" else None)
    torch.cuda.synchronize()
    res = {"status": int(out["status"].item()), "rgb": out["rgb"].cpu().numpy(), "T": out["T"].cpu().numpy(),
           "last": out["last"].cpu().numpy(), "pairs": int(r.pair_count().item()),
           "contrib": int(r.stats()[1].item()), "redone": int(r.stats()[2].item()),
           "score": score.cpu().numpy() if score is not None else None,
           "loss": float(out["loss"].item()) if out["loss"] is not None else None}
    if grads is not None:
        res["grads"] = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}
    return res


def oracle_views(g, cams, edges=None):
    outs = []
    for v, cam in enumerate(cams):
        outs.append(orc.render(g, cam, edge=None if edges is None else edges[v]))
    return outs


def exempt_gaussians(g, cam, ref, window=GATE_REL):
    """Indices of Gaussians whose footprint holds a gate-exempt pixel."""
    ys, xs = np.nonzero(ref["gate_gap"] < window)
    proj = ref["proj"]
    out = set()
    for x, y in zip(xs, ys):
        d = np.hypot(proj[:, orc.P_MX] - (x + 0.5), proj[:, orc.P_MY] - (y + 0.5))
        hit = (proj[:, orc.P_VALID] > 0) & (proj[:, orc.P_RADIUS] >= 0) & (d <= proj[:, orc.P_RADIUS] + 1)
        out.update(np.nonzero(hit)[0].tolist())
    return out


def check_image(res, refs, cams):
    """RGB and T_final within 1e-4 outside the gate-exempt pixels, whose count
    must stay within EXEMPT_FRAC of the pixels compared; returns that count."""
    off = 0
    n_ex = n_px = 0
    for cam, ref in zip(cams, refs):
        h, w = cam["height"], cam["width"]
        rgb = res["rgb"][off:off + h * w].reshape(h, w, 3)
        T = res["T"][off:off + h * w].reshape(h, w)
        ok = ref["gate_gap"] >= GATE_REL
        n_ex += int((~ok).sum())
        n_px += h * w
        err = np.abs(rgb - ref["rgb"]).max(axis=2)
        assert err[ok].max(initial=0) <= 1e-4, err[ok].max()
        assert np.abs(T - ref["T"])[ok].max(initial=0) <= 1e-4
        off += h * w
    assert n_ex <= EXEMPT_FRAC * n_px, (n_ex, n_px)
    return n_ex


def check_scores(s_gpu, s_ref, skip=()):
    keep = np.ones(s_ref.shape[0], bool)
    keep[list(skip)] = False
    floor = 1e-3 * np.abs(s_ref).max(initial=0)
    rel = np.abs(s_gpu - s_ref) / np.maximum(np.abs(s_ref), max(floor, 1e-30))
    assert rel[keep].max(initial=0) <= 1e-4, rel[keep].max()


def check_grads(gr_gpu, gr_ref, gr_mag, n, skip=()):
    """Every entry of every group within conftest.grad_bound, outside the
    gate-exempt Gaussians; gr_mag is the oracle's magnitude adjoint."""
    keep = np.ones(n, bool)
    keep[list(skip)] = False
    for name in GROUPS:
        a = gr_gpu[name][:n].reshape(n, -1)
        b = gr_ref[name].reshape(n, -1)
        mag = gr_mag[name].reshape(n, -1)
        assert_grads_match(name, a[keep], b[keep], mag[keep])


def test_tiny_config_matches_oracle(gsp_lib):
    g = synth.gaussians(2000, 0, seed=1)
    cam = synth.camera_front(128, 128)
    tgt = synth.image(128, 128, 2000)
    e = oe.edge_map(tgt)["E"]
    res = gpu_render(gsp_lib, g, [cam], targets=[tgt], edges=[e])
    assert res["status"] == 0
    ref = orc.render(g, cam, edge=e)
    check_image(res, [ref], [cam])
    # composited (pixel, Gaussian) pairs: exact outside gate-exempt pixels
    ex = ref["gate_gap"] < GATE_REL
    assert abs(res["contrib"] - int(ref["ncontrib"].sum())) <= int(ref["ncontrib"][ex].sum()) + int(ex.sum())
    check_scores(res["score"], ref["score"], exempt_gaussians(g, cam, ref))
    loss_ref, _ = orc.l1_loss(ref["rgb"], tgt)
    assert abs(res["loss"] - loss_ref) <= 1e-5 * loss_ref


@pytest.mark.parametrize("seed", range(6))
def test_tiny_scenes_against_brute_force(gsp_lib, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 65))
    g = synth.gaussians(n, [0, 1, 2, 3][seed % 4], seed=500 + seed)
    g["log_scales"] += np.float32(rng.uniform(0.0, 1.5))
    w, h = int(rng.integers(16, 49)), int(rng.integers(16, 49))
    cam = synth.camera_look_at(rng.uniform(-1, 1, 3) + np.array([0, 0, -4.0]), w, h)
    e = rng.uniform(0, 3, (h, w))
    res = gpu_render(gsp_lib, g, [cam], edges=[e])
    ref = orc.render(g, cam, edge=e, brute=True)
    check_image(res, [ref], [cam])
    ex = ref["gate_gap"] < GATE_REL
    assert abs(res["contrib"] - int(ref["ncontrib"].sum())) <= int(ref["ncontrib"][ex].sum()) + int(ex.sum())
    check_scores(res["score"], ref["score"], exempt_gaussians(g, cam, ref))


def test_uneven_views_in_one_launch(gsp_lib):
    g = synth.gaussians(800, 3, seed=8)
    g["log_scales"] += np.float32(0.7)
    sizes = [(80, 60), (128, 128), (194, 102)]
    cams = [synth.camera_ring(k, 3, resolutions=sizes) for k in range(3)]
    rng = np.random.default_rng(3)
    edges = [rng.uniform(0, 2, (c["height"], c["width"])) for c in cams]
    res = gpu_render(gsp_lib, g, cams, edges=edges)
    refs = oracle_views(g, cams, edges)
    check_image(res, refs, cams)
    skip = set()
    for c, r in zip(cams, refs):
        skip |= exempt_gaussians(g, c, r)
    check_scores(res["score"], sum(r["score"] for r in refs), skip)


def test_empty_and_fully_culled_scenes(gsp_lib):
    cam = synth.camera_front(40, 24)
    g = synth.gaussians(0, 0)
    res = gpu_render(gsp_lib, g, [cam], edges=[np.ones((24, 40))], capacity=16)
    assert res["status"] == 0 and np.all(res["rgb"] == 0) and np.all(res["T"] == 1) and res["pairs"] == 0
    g = synth.gaussians(50, 0, seed=2)
    g["means"][:, 2] = -5.0  # behind the camera
    res = gpu_render(gsp_lib, g, [cam], edges=[np.ones((24, 40))])
    assert np.all(res["rgb"] == 0) and np.all(res["score"] == 0) and res["pairs"] == 0


def test_pair_capacity_overflow_is_reported_and_writes_nothing(gsp_lib):
    import torch
    g = synth.gaussians(2000, 0, seed=1)
    cam = synth.camera_front(128, 128)
    gs = gsp_lib.GaussianSet.from_arrays(g)
    r = gsp_lib.Renderer(gs, [cam], pair_capacity=100)
    sentinel = {"rgb": torch.full((128 * 128, 3), -7.0, device="cuda"),
                "T": torch.full((128 * 128,), -7.0, device="cuda"),
                "last": torch.full((128 * 128,), -7, dtype=torch.int32, device="cuda")}
    out = r.forward(out=sentinel)
    torch.cuda.synchronize()
    assert int(out["status"].item()) == gsp_lib._lib.GSP_ERR_CAPACITY
    assert bool((out["rgb"] == -7).all()) and bool((out["T"] == -7).all())
    assert int(r.pair_count().item()) > 100


def _grad_scene():
    rng = np.random.default_rng(5)
    g = synth.gaussians(40, 3, seed=3)
    g["log_scales"] = (g["log_scales"] + 1.2).astype(np.float32)
    g["quats"] = (g["quats"] * rng.uniform(0.5, 2.0, (40, 1))).astype(np.float32)
    return g, synth.camera_look_at((0.5, -0.3, -4.0), 48, 40), synth.image(40, 48, 2000)


def test_gradients_match_oracle_adjoint(gsp_lib):
    g, cam, _ = _grad_scene()
    rng = np.random.default_rng(11)
    dL = rng.normal(size=(40 * 48, 3)) / (40 * 48)
    res = gpu_render(gsp_lib, g, [cam], dL=dL)
    ref = orc.render(g, cam)
    gr = orc.render_bwd(g, cam, dL.reshape(40, 48, 3))
    gm = orc.render_bwd(g, cam, dL.reshape(40, 48, 3), magnitude=True)
    check_grads(res["grads"], gr, gm, 40, exempt_gaussians(g, cam, ref))


def test_gradients_match_central_differences(gsp_lib):
    g, cam, tgt = _grad_scene()
    res = gpu_render(gsp_lib, g, [cam], targets=[tgt])
    ref = orc.render(g, cam)
    # pixels with contributors whose C is within 1e-5 of the target could take
    # their L1 sign differently (empty pixels are exactly 0 on both sides)
    t = tgt / 255.0
    exact = (ref["rgb"] == 0.0) & (t == 0.0)  # clamped colour against black: 0 on both sides
    near = ((np.abs(ref["rgb"] - t) < 1e-5) & ~exact).any(axis=2)
    assert near.sum() == 0
    items = [(i, n, c) for i in range(40) for n, k in zip(GROUPS, (3, 3, 4, 1, 48)) for c in range(k)]
    fd1, fd2 = orc.fd_grad(g, cam, tgt, items)
    kink = np.abs(fd1 - fd2) > 0.1 * np.maximum(np.abs(fd1), 1e-12)
    an = np.array([res["grads"][n][i].ravel()[c] if res["grads"][n].ndim > 1 else res["grads"][n][i]
                   for (i, n, c) in items])
    skip = exempt_gaussians(g, cam, ref)
    for name in GROUPS:
        sel = np.array([it[1] == name and it[0] not in skip for it in items]) & ~kink
        rms = np.sqrt(np.mean(fd1[sel] ** 2))
        rel = np.abs(an[sel] - fd1[sel]) / np.maximum(np.abs(fd1[sel]), 1e-3 * rms)
        assert rel.max() <= 1e-3, (name, rel.max())


def test_l1_sign_map_equals_explicit_upstream_gradient(gsp_lib):
    g, cam, tgt = _grad_scene()
    a = gpu_render(gsp_lib, g, [cam], targets=[tgt])
    t32 = tgt.reshape(-1, 3).astype(np.float32) / np.float32(255.0)  # IEEE FP32 division, as on the device
    diff = a["rgb"].astype(np.float64) - t32.astype(np.float64)
    dL = np.sign(diff) / diff.size
    # exact ties (empty pixels against black) have sign 0 on both paths
    assert ((np.abs(diff) < 1e-6) & (diff != 0)).sum() == 0
    b = gpu_render(gsp_lib, g, [cam], dL=dL)
    # the two runs sum the same FP32 terms in unspecified (atomic) order
    for name in GROUPS:
        scale = np.sqrt(np.mean(a["grads"][name] ** 2))
        np.testing.assert_allclose(a["grads"][name], b["grads"][name], rtol=1e-5, atol=1e-6 * scale)


def test_score_in_backward_equals_score_in_forward(gsp_lib):
    g = synth.gaussians(2000, 0, seed=1)
    cam = synth.camera_front(128, 128)
    tgt = synth.image(128, 128, 2000)
    e = oe.edge_map(tgt)["E"]
    a = gpu_render(gsp_lib, g, [cam], targets=[tgt], edges=[e], score_in="fwd")
    b = gpu_render(gsp_lib, g, [cam], targets=[tgt], edges=[e], score_in="bwd")
    check_scores(b["score"], a["score"].astype(np.float64))


def test_capacity_rows_beyond_count_are_ignored(gsp_lib):
    g = synth.gaussians(300, 1, seed=4)
    cam = synth.camera_front(64, 48)
    a = gpu_render(gsp_lib, g, [cam], edges=[np.ones((48, 64))])
    b = gpu_render(gsp_lib, g, [cam], edges=[np.ones((48, 64))], capacity=1000)
    assert np.array_equal(a["rgb"], b["rgb"])
    np.testing.assert_allclose(a["score"], b["score"][:300], rtol=1e-5, atol=1e-7)
    assert np.all(b["score"][300:] == 0)


def test_positional_statistic_matches_oracle(gsp_lib):
    """The positional statistic of the gradient-threshold masking, accumulated by
    the adjoint over three uneven views and two calls, against the oracle's
    screen-space mean gradients: counts exact and sums within 1e-4 relative
    (floor 1e-3 x RMS) plus the rounding bound 64 u A (A: the norm of the
    mean gradient's magnitude adjoint, summed over the views), outside the
    gate-exempt Gaussians."""
    import torch
    n = 1500
    g = synth.gaussians(n, 3, seed=31)
    g["log_scales"] += np.float32(0.6)
    sizes = [(80, 60), (64, 64), (97, 51)]
    cams = [synth.camera_ring(k, 3, resolutions=sizes) for k in range(3)]
    npix = sum(c["width"] * c["height"] for c in cams)
    rng = np.random.default_rng(17)
    dL = rng.normal(size=(npix, 3)) / npix
    dL[rng.uniform(size=npix) < 0.2] = 0.0  # pixels without upstream gradient
    gs = gsp_lib.GaussianSet.from_arrays(g)
    r = gsp_lib.Renderer(gs, cams, 1 << 22)
    out = r.forward()
    psum = torch.zeros(gs.capacity, device="cuda")
    pcnt = torch.zeros(gs.capacity, dtype=torch.int32, device="cuda")
    dl_t = torch.from_numpy(dL.astype(np.float32)).cuda()
    r.backward(out, dL_drgb=dl_t, pos_grad=(psum, pcnt))
    torch.cuda.synchronize()
    s1, c1 = psum.cpu().numpy().astype(np.float64), pcnt.cpu().numpy()
    r.backward(out, dL_drgb=dl_t, pos_grad=(psum, pcnt))
    torch.cuda.synchronize()
    s2, c2 = psum.cpu().numpy().astype(np.float64), pcnt.cpu().numpy()
    assert int(out["status"].item()) == 0
    views, skip, off = [], set(), 0
    mag = np.zeros(n)
    for cam in cams:
        w, h = cam["width"], cam["height"]
        ref = orc.render(g, cam)
        dlv = dL[off:off + w * h].reshape(h, w, 3)
        views.append(orc.render_bwd(g, cam, dlv, proj=ref["proj"])["g2d"])
        gm = orc.render_bwd(g, cam, dlv, proj=ref["proj"], magnitude=True)["g2d"]
        mag += np.hypot(gm[:, 0], gm[:, 1])
        skip |= exempt_gaussians(g, cam, ref)
        off += w * h
    s_ref, c_ref = od.pos_grad_stats(views)
    keep = np.ones(n, bool)
    keep[list(skip)] = False
    assert keep.sum() > n // 2 and (c_ref[keep] > 0).sum() > 300
    assert np.array_equal(c1[:n][keep], c_ref[keep])
    rms = np.sqrt(np.mean(s_ref[keep] ** 2))
    assert_grads_match("pos_grad_sum", s1[:n][keep], s_ref[keep], mag[keep], rms)
    # a second call adds the same statistic again
    assert np.array_equal(c2, 2 * c1)
    np.testing.assert_allclose(s2, 2 * s1, rtol=1e-5, atol=1e-6 * rms)


def test_footprints_wider_than_255_tiles_and_taller_than_16_rows(gsp_lib):
    """A 4400 x 320 view (275 x 20 tiles) with Gaussians whose footprints span
    more than 255 tiles across (their per-row column intervals are not stored:
    every row keeps the full rectangle) and more than 16 tile rows (rows past
    the 16 stored intervals keep the full width), beside small ones: RGB, T
    and every gradient against the oracle."""
    rng = np.random.default_rng(17)
    n_big, n_small = 12, 48
    n = n_big + n_small
    g = synth.gaussians(n, 1, seed=23)
    g["means"][:n_big] = rng.uniform([-0.3, -0.05, -0.3], [0.3, 0.05, 0.3], (n_big, 3)).astype(np.float32)
    g["log_scales"][:n_big] = np.stack([rng.uniform(-0.1, 0.15, n_big), rng.uniform(-2.6, -1.6, n_big),
                                        rng.uniform(-2.0, -1.0, n_big)], axis=1).astype(np.float32)
    g["opacity_logits"][:n_big] = rng.uniform(-2.5, -1.0, g["opacity_logits"][:n_big].shape).astype(np.float32)
    cam = synth.camera_front(4400, 320)
    w, h = cam["width"], cam["height"]
    dL = rng.normal(size=(h * w, 3)) / (h * w)
    res = gpu_render(gsp_lib, g, [cam], dL=dL, pair_capacity=1 << 22)
    assert res["status"] == 0
    ref = orc.render(g, cam)
    proj = ref["proj"]
    tiles_x = (w + 15) // 16
    wide = np.minimum(proj[:n_big, orc.P_TX1], tiles_x - 1) - np.maximum(proj[:n_big, orc.P_TX0], 0) + 1
    tall = np.minimum(proj[:n_big, orc.P_TY1], (h + 15) // 16 - 1) - np.maximum(proj[:n_big, orc.P_TY0], 0) + 1
    valid = proj[:n_big, orc.P_VALID] > 0
    assert (valid & (wide > 255)).sum() >= 3, wide  # rectangles wider than 255 tiles
    assert (valid & (tall > 16)).sum() >= 3, tall   # and taller than 16 tile rows
    check_image(res, [ref], [cam])
    gr = orc.render_bwd(g, cam, dL.reshape(h, w, 3))
    gm = orc.render_bwd(g, cam, dL.reshape(h, w, 3), magnitude=True)
    check_grads(res["grads"], gr, gm, n, exempt_gaussians(g, cam, ref))


def test_degenerate_view_shapes_in_one_batch(gsp_lib):
    """One launch over views of 1 x 1, 3 x 250, 250 x 3, 17 x 17 and 160 x 120
    pixels (single tiles, single tile rows and columns, ragged tails): RGB, T,
    edge scores and every gradient against the oracle, summed over the views."""
    sizes = [(1, 1), (250, 3), (3, 250), (17, 17), (160, 120)]
    g = synth.gaussians(400, 2, seed=29)
    g["log_scales"] += np.float32(0.5)
    n = 400
    cams = [synth.camera_ring(k, len(sizes), resolutions=sizes) for k in range(len(sizes))]
    rng = np.random.default_rng(5)
    edges = [rng.uniform(0, 2, (c["height"], c["width"])) for c in cams]
    npix = sum(c["width"] * c["height"] for c in cams)
    dL = rng.normal(size=(npix, 3)) / npix
    res = gpu_render(gsp_lib, g, cams, edges=edges, dL=dL, score_in="bwd")
    assert res["status"] == 0
    refs = oracle_views(g, cams, edges)
    check_image(res, refs, cams)
    skip = set()
    gr = {k: 0.0 for k in GROUPS}
    gm = {k: 0.0 for k in GROUPS}
    off = 0
    for c, r in zip(cams, refs):
        h, w = c["height"], c["width"]
        skip |= exempt_gaussians(g, c, r)
        d = dL[off:off + h * w].reshape(h, w, 3)
        a = orc.render_bwd(g, c, d, proj=r["proj"])
        m = orc.render_bwd(g, c, d, proj=r["proj"], magnitude=True)
        for k in GROUPS:
            gr[k] = gr[k] + a[k].reshape(n, -1)
            gm[k] = gm[k] + m[k].reshape(n, -1)
        off += h * w
    check_scores(res["score"], sum(r["score"] for r in refs), skip)
    check_grads(res["grads"], gr, gm, n, skip)


@pytest.mark.parametrize("prefix", [1, 7, 64])
def test_tile_list_prefix_and_redo_leave_results_unchanged(gsp_lib, prefix):
    """Only the first list_prefix entries of each tile list are written before
    the forward compositing; tiles that need more save their pixels' state,
    get the rest of their list and resume.  The forward's outputs are bitwise
    those of whole lists, the gradients (score in the adjoint) still match
    the oracle, and the resumed tiles are counted."""
    g = synth.gaussians(800, 3, seed=8)
    g["log_scales"] += np.float32(0.7)
    g["opacity_logits"] -= np.float32(2.0)  # few pixels saturate: many tiles need their whole list
    sizes = [(80, 60), (128, 128), (194, 102)]
    cams = [synth.camera_ring(k, 3, resolutions=sizes) for k in range(3)]
    rng = np.random.default_rng(3)
    edges = [rng.uniform(0, 2, (c["height"], c["width"])) for c in cams]
    npix = sum(c["width"] * c["height"] for c in cams)
    dL = rng.normal(size=(npix, 3)) / npix
    whole = gpu_render(gsp_lib, g, cams, edges=edges, dL=dL, score_in="bwd", list_prefix=1 << 40)
    part = gpu_render(gsp_lib, g, cams, edges=edges, dL=dL, score_in="bwd", list_prefix=prefix)
    assert whole["status"] == 0 and part["status"] == 0
    assert whole["redone"] == 0 and part["redone"] > 0
    for k in ("rgb", "T", "last"):
        assert np.array_equal(part[k], whole[k]), k
    assert part["contrib"] == whole["contrib"] and part["pairs"] == whole["pairs"]
    refs = oracle_views(g, cams, edges)
    check_image(part, refs, cams)
    skip = set()
    for c, r in zip(cams, refs):
        skip |= exempt_gaussians(g, c, r)
    check_scores(part["score"], sum(r["score"] for r in refs), skip)
    off = 0
    gr, gm = {}, {}
    for c in cams:
        n_c = c["width"] * c["height"]
        d = dL[off:off + n_c].reshape(c["height"], c["width"], 3)
        a = orc.render_bwd(g, c, d)
        b = orc.render_bwd(g, c, d, magnitude=True)
        for k in a:
            gr[k] = gr.get(k, 0) + a[k]
            gm[k] = gm.get(k, 0) + b[k]
        off += n_c
    check_grads(part["grads"], gr, gm, 800, skip)


def test_score_in_forward_with_resumed_tiles(gsp_lib):
    """The forward's edge score over resumed tiles: each (pixel, Gaussian)
    term is added once, before or after the resume."""
    g = synth.gaussians(800, 3, seed=8)
    g["opacity_logits"] -= np.float32(2.0)
    cam = synth.camera_front(128, 96)
    e = np.random.default_rng(4).uniform(0, 2, (96, 128))
    a = gpu_render(gsp_lib, g, [cam], edges=[e], score_in="fwd", list_prefix=5)
    b = gpu_render(gsp_lib, g, [cam], edges=[e], score_in="fwd", list_prefix=1 << 40)
    assert a["redone"] > 0 and b["redone"] == 0
    for k in ("rgb", "T", "last"):
        assert np.array_equal(a[k], b[k]), k
    # floating-point atomics: equal up to the order of the additions
    assert np.allclose(a["score"], b["score"], rtol=1e-5, atol=1e-6 * float(np.abs(b["score"]).max()))
    ref = orc.render(g, cam, edge=e)
    check_image(a, [ref], [cam])
    check_scores(a["score"], ref["score"], exempt_gaussians(g, cam, ref))
