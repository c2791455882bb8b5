"""Full-size parity: 1,000,000 SH-3 Gaussians on one 1237x822 view, in the
launch configuration the benchmark times (capacity N + 10 %, one call over the
whole view), checked on sampled outputs the FP64 oracle computes directly.

* RGB and T_final on three 32x32 pixel regions (tile-aligned at the centre,
  unaligned, and the ragged bottom-right tiles) within 1e-4 absolute.
* Per-Gaussian edge scores within 1e-4 relative for every Gaussian: the edge
  map is the oracle's, kept on the regions and zero elsewhere, so the score
  is exactly the sum the oracle's region renders give.
* The score invariant at full size: with E = 1 the scores sum to sum(1 - T).
* Gradients of every Gaussian against the oracle's analytic adjoint for an
  upstream gradient that lives on one region, entry by entry: 1e-4 relative
  (floor 1e-3 x the group RMS) plus the FP32 rounding bound of cancelling
  sums (conftest.grad_bound).
* Central finite differences of the L1 loss restricted to 25 separated
  regions, on a 1,000-Gaussian subset x 8 scalars, within 1e-3 relative
  (kinks excluded).
Pixels at which the oracle meets a gate within GATE_REL are exempt, and so
are the Gaussians whose results such a flip would move; they must stay within
EXEMPT_FRAC of the pixels compared.
"""
import concurrent.futures as cf
import multiprocessing as mp
import os

import numpy as np
import pytest

import synth
from conftest import EXEMPT_FRAC, GATE_REL, assert_grads_match
from oracle import edge as oe
from oracle import raster as orc

pytestmark = pytest.mark.gpu

N, W, H = 1_000_000, 1237, 822
CAP = N + N // 10
REGIONS = [(608, 400, 640, 432), (477, 253, 509, 285), (1205, 790, 1237, 822)]
GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")
FD_SCALARS = [("means", 0), ("means", 2), ("log_scales", 0), ("quats", 0), ("quats", 2), ("opacity_logits", 0),
              ("sh", 0), ("sh", 45)]


@pytest.fixture(scope="module")
def scene():
    g = synth.gaussians(N, 3, seed=1)
    cam = synth.camera_front(W, H)
    tgt = synth.image(H, W, 2000)
    proj = orc.project(g, cam)
    order = orc.order(proj)
    return g, cam, tgt, proj, order


def _renderer(gsp, g, cam):
    import torch
    gs = gsp.GaussianSet.from_arrays(g, capacity=CAP)
    probe = gsp.Renderer(gs, [cam], pair_capacity=1 << 27)
    probe.forward()
    torch.cuda.synchronize()
    pairs = int(probe.pair_count().item())
    del probe
    return gs, gsp.Renderer(gs, [cam], pair_capacity=int(pairs * 1.05) + 1024)


def _exempt_gaussians(proj, order, gap):
    ex = gap < GATE_REL
    if not ex.any():
        return np.zeros(proj.shape[0], bool)
    return orc.gate_affected(proj, ex, GATE_REL, order)


def test_1m_regions_rgb_T_and_every_score(gsp_lib, scene):
    import torch
    g, cam, tgt, proj, order = scene
    e_full = oe.edge_map(tgt)["E"]
    e_reg = np.zeros((H, W))
    for (x0, y0, x1, y1) in REGIONS:
        e_reg[y0:y1, x0:x1] = e_full[y0:y1, x0:x1]
    e32 = e_reg.astype(np.float32)
    gs, r = _renderer(gsp_lib, g, cam)
    score = torch.zeros(CAP, device="cuda")
    t_gpu = torch.from_numpy(tgt).cuda()
    out = r.forward(targets=[t_gpu], edge=torch.from_numpy(e32.ravel()).cuda(), score=score)
    torch.cuda.synchronize()
    assert int(out["status"].item()) == 0
    rgb = out["rgb"].cpu().numpy().reshape(H, W, 3)
    T = out["T"].cpu().numpy().reshape(H, W)
    s_ref = np.zeros(N)
    gap = np.full((H, W), np.inf)
    n_ex = n_px = 0
    for reg in REGIONS:
        x0, y0, x1, y1 = reg
        ref = orc.render(g, cam, edge=e32.astype(np.float64), region=reg, proj=proj, order=order)
        ok = ref["gate_gap"][y0:y1, x0:x1] >= GATE_REL
        n_ex += int((~ok).sum())
        n_px += ok.size
        err = np.abs(rgb[y0:y1, x0:x1] - ref["rgb"][y0:y1, x0:x1]).max(axis=2)
        assert err[ok].max(initial=0) <= 1e-4
        assert np.abs(T[y0:y1, x0:x1] - ref["T"][y0:y1, x0:x1])[ok].max(initial=0) <= 1e-4
        s_ref += ref["score"]
        gap[y0:y1, x0:x1] = ref["gate_gap"][y0:y1, x0:x1]
    assert n_ex <= EXEMPT_FRAC * n_px, (n_ex, n_px)
    assert np.all(rgb[790:, 1205:] == 0) and np.all(T[790:, 1205:] == 1)  # outside the scene
    skip = _exempt_gaussians(proj, order, gap)
    s_gpu = score.cpu().numpy()[:N].astype(np.float64)
    assert np.all(score.cpu().numpy()[N:] == 0)
    floor = 1e-3 * np.abs(s_ref).max()
    rel = np.abs(s_gpu - s_ref) / np.maximum(np.abs(s_ref), floor)
    assert (s_ref > 0).sum() > 200  # pixels saturate after ~65 Gaussians: a few hundred reach the regions
    assert rel[~skip].max() <= 1e-4, rel[~skip].max()


def test_1m_score_invariant_with_unit_edge_map(gsp_lib, scene):
    import torch
    g, cam, _, _, _ = scene
    gs, r = _renderer(gsp_lib, g, cam)
    score = torch.zeros(CAP, device="cuda", dtype=torch.float32)
    out = r.forward(edge=torch.ones(W * H, device="cuda"), score=score)
    torch.cuda.synchronize()
    lhs = float(score.double().sum().item())
    rhs = float((1.0 - out["T"].double()).sum().item())
    assert abs(lhs - rhs) <= 1e-4 * rhs


def test_1m_region_gradients_match_oracle_adjoint(gsp_lib, scene):
    import torch
    g, cam, _, proj, order = scene
    x0, y0, x1, y1 = REGIONS[0]
    dl = np.zeros((H, W, 3))
    dl[y0:y1, x0:x1] = np.random.default_rng(4).normal(size=(y1 - y0, x1 - x0, 3)) / (W * H)
    gs, r = _renderer(gsp_lib, g, cam)
    out = r.forward()
    grads = r.backward(out, dL_drgb=torch.from_numpy(dl.astype(np.float32).reshape(-1, 3)).cuda())
    torch.cuda.synchronize()
    ref = orc.render(g, cam, region=REGIONS[0], proj=proj, order=order)
    dl64 = dl.astype(np.float32).astype(np.float64)
    gr = orc.render_bwd(g, cam, dl64, proj=proj, region=REGIONS[0])
    gm = orc.render_bwd(g, cam, dl64, proj=proj, region=REGIONS[0], magnitude=True)
    x0, y0, x1, y1 = REGIONS[0]
    assert (ref["gate_gap"][y0:y1, x0:x1] < GATE_REL).sum() <= EXEMPT_FRAC * (x1 - x0) * (y1 - y0)
    skip = _exempt_gaussians(proj, order, ref["gate_gap"])
    touched = np.abs(gr["opacity_logits"]) > 0
    assert touched.sum() > 100
    keep = touched & ~skip
    for name in GROUPS:
        a = grads[name][:N].cpu().numpy().astype(np.float64).reshape(N, -1)
        b = gr[name].reshape(N, -1)
        assert np.all(a[~touched & ~skip] == 0)
        assert_grads_match(name, a[keep], b[keep], gm[name].reshape(N, -1)[keep])


def _fd_chunk(args):
    g_sub, cam, tgt, proj_sub, mask, items, scale = args
    fd1, fd2 = orc.fd_grad(g_sub, cam, tgt, items, rel_h=FD_REL_H, proj=proj_sub, loss_mask=mask)
    return fd1 * scale, fd2 * scale


def crop_scene(g, cam, region):
    """The scene as the pixels of region see it, for the oracle: a crop camera
    (same intrinsics, principal point moved by the region's origin, image the
    size of the region) and the Gaussians that can reach those pixels - their
    footprint touches the region and they lie in front of the depth at which
    every pixel of the region has stopped compositing.  The cut is accepted
    only if the crop composites identically with and without it."""
    x0, y0, x1, y1 = region
    crop = dict(cam, cx=float(cam["cx"]) - x0, cy=float(cam["cy"]) - y0, width=x1 - x0, height=y1 - y0)
    pc = orc.project(g, crop)
    rad = pc[:, orc.P_RADIUS] + 2.0
    near = ((pc[:, orc.P_VALID] > 0) & (pc[:, orc.P_RADIUS] >= 0) & (pc[:, orc.P_MX] + rad >= 0) &
            (pc[:, orc.P_MX] - rad <= x1 - x0) & (pc[:, orc.P_MY] + rad >= 0) & (pc[:, orc.P_MY] - rad <= y1 - y0))
    sub = np.nonzero(near)[0]

    def take(idx):
        return ({k: (v[idx] if isinstance(v, np.ndarray) else v) for k, v in g.items()},
                np.ascontiguousarray(pc[idx]))

    g1, p1 = take(sub)
    o1 = orc.order(p1)
    full = orc.render(g1, crop, proj=p1, order=o1)
    pos = np.full(sub.size, -1)
    pos[o1] = np.arange(o1.size)
    lastpos = int(pos[full["last_id"][full["last_id"] >= 0]].max(initial=-1))
    if (full["T"] > 1e-3).any():  # a pixel that never stops sees every Gaussian
        lastpos = o1.size - 1
    cut = min(o1.size, lastpos + max(64, lastpos // 10) + 1)
    sub2 = sub[np.sort(o1[:cut])]
    g2, p2 = take(sub2)
    again = orc.render(g2, crop, proj=p2)
    for key in ("rgb", "T", "ncontrib"):
        assert np.array_equal(full[key], again[key])
    return crop, sub2, g2, p2


def fd_on_regions(g, cam, tgt, mask, items_by_region, workers):
    """Central differences (h and h/2) of the L1 loss summed over mask,
    normalised by the full view's 3 W H.  items_by_region lists, per region,
    the (index, name, component) items whose Gaussian reaches that region; the
    loss is a sum over the regions, so an item's differences are summed over
    the regions it reaches."""
    tasks, slots = [], []
    for region, items in items_by_region:
        if not items:
            continue
        x0, y0, x1, y1 = region
        crop, sub, g2, p2 = crop_scene(g, cam, region)
        local = [(int(np.searchsorted(sub, i)), n, c) for (i, n, c) in items]
        assert all(sub[j] == it[0] for (j, _, _), it in zip(local, items))
        scale = float((x1 - x0) * (y1 - y0)) / float(cam["width"] * cam["height"])
        k = max(1, (len(local) + 63) // 64)
        for c in range(k):
            tasks.append((g2, crop, tgt[y0:y1, x0:x1], p2, mask[y0:y1, x0:x1], local[c::k], scale))
            slots.append([it for it in items[c::k]])
    if workers > 1:
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            parts = list(ex.map(_fd_chunk, tasks))
    else:
        parts = [_fd_chunk(t) for t in tasks]
    out = {}
    for its, (a, b) in zip(slots, parts):
        for it, x, y in zip(its, a, b):
            px, py = out.get(it, (0.0, 0.0))
            out[it] = (px + x, py + y)
    return out


FD_OFFSETS = (-200, -100, 0, 100, 200)
FD_REL_H = 1e-7  # 1M Gaussians: a 1e-5 depth step would cross several neighbours' depths


def test_1m_finite_differences_on_a_1000_gaussian_subset(gsp_lib, scene):
    """1,000 Gaussians x 8 scalars; the loss is the L1 loss summed over 25
    separated 32x32 regions."""
    import torch
    g, cam, tgt, proj, order = scene
    cx, cy = W // 2, H // 2
    regions = [(cx + dx - 16, cy + dy - 16, cx + dx + 16, cy + dy + 16) for dy in FD_OFFSETS for dx in FD_OFFSETS]
    t = tgt / 255.0
    mask = np.zeros((H, W), bool)
    gap = np.full((H, W), np.inf)
    refs = []
    for reg in regions:
        x0, y0, x1, y1 = reg
        ref = orc.render(g, cam, region=reg, proj=proj, order=order)
        refs.append(ref)
        mask[y0:y1, x0:x1] = True
        gap[y0:y1, x0:x1] = ref["gate_gap"][y0:y1, x0:x1]
        # pixels whose colour is within 1e-5 of the target: their L1 sign is not fixed
        mask[y0:y1, x0:x1] &= ~(np.abs(ref["rgb"][y0:y1, x0:x1] - t[y0:y1, x0:x1]) < 1e-5).any(axis=2)
    assert (gap[mask] < GATE_REL).sum() <= EXEMPT_FRAC * mask.sum()
    mask &= gap >= GATE_REL
    skip = _exempt_gaussians(proj, order, gap)
    gs, r = _renderer(gsp_lib, g, cam)
    out = r.forward()
    torch.cuda.synchronize()
    rgb = out["rgb"].cpu().numpy().reshape(H, W, 3).astype(np.float64)
    t32 = (tgt.astype(np.float32) / np.float32(255.0)).astype(np.float64)
    dl = np.sign(rgb - t32) / (3.0 * W * H) * mask[:, :, None]
    grads = r.backward(out, dL_drgb=torch.from_numpy(dl.astype(np.float32).reshape(-1, 3)).cuda())
    torch.cuda.synchronize()
    gh = {n: grads[n][:N].cpu().numpy().reshape(N, -1).astype(np.float64) for n in GROUPS}
    # the Gaussians each region's loss depends on (non-zero oracle opacity gradient)
    hits = []
    for reg in regions:
        x0, y0, x1, y1 = reg
        dlr = np.zeros_like(dl)
        dlr[y0:y1, x0:x1] = dl[y0:y1, x0:x1]
        gr = orc.render_bwd(g, cam, dlr.astype(np.float32).astype(np.float64), proj=proj, region=reg)
        hits.append(np.abs(gr["opacity_logits"]) > 0)
    reach = np.any(hits, axis=0)
    cand = np.nonzero(reach & ~skip)[0]
    pick = np.sort(np.random.default_rng(9).choice(cand, size=min(1000, cand.size), replace=False))
    assert pick.size == 1000
    items = [(int(i), n, c) for i in pick for (n, c) in FD_SCALARS]
    items_by_region = [(reg, [it for it in items if hit[it[0]]]) for reg, hit in zip(regions, hits)]
    workers = max(1, min(16, os.cpu_count() or 1))
    fd = fd_on_regions(g, cam, tgt, mask, items_by_region, workers)
    fd1 = np.array([fd[it][0] for it in items])
    fd2 = np.array([fd[it][1] for it in items])
    kink = np.abs(fd1 - fd2) > 0.1 * np.maximum(np.abs(fd1), 1e-12)
    assert kink.sum() < 0.05 * len(items)
    an = np.array([gh[n][i, c] for (i, n, c) in items])
    for name in GROUPS:
        sel = np.array([it[1] == name for it in items]) & ~kink
        rms = np.sqrt(np.mean(fd1[sel] ** 2))
        rel = np.abs(an[sel] - fd1[sel]) / np.maximum(np.abs(fd1[sel]), 1e-3 * rms)
        assert rel.max() <= 1e-3, (name, rel.max())
