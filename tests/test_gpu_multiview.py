"""Batched multi-view parity: 3,000,000 SH-3 Gaussians and 8 ring cameras of
uneven resolution (640x480 ... 1920x1080) in one forward and one adjoint call,
captured as a CUDA graph, with the compositing variants the autotuner picks.

Checked on sampled outputs the FP64 oracle computes directly: RGB and T_final
(1e-4 absolute) on a 32x32 region of every view, the per-Gaussian edge score
summed over the views (1e-4 relative, every Gaussian; the edge map lives on
the regions), and every gradient entry for an upstream gradient on those
regions (1e-4 relative, floor 1e-3 x the RMS of the group, plus the FP32
rounding bound of cancelling sums: conftest.grad_bound) view by view, the
batched launch given an upstream gradient on one view at a time; the
all-view gradient must then match the sum of the per-view ones by the same
criterion (both are FP32 sums of the same terms in different orders).  Gate-
exempt pixels stay within EXEMPT_FRAC of the pixels compared.  Also: the compositing variants agree with each other, and
a graph replay reproduces the eager results bit for bit.
"""
import numpy as np
import pytest

import synth
from conftest import EXEMPT_FRAC, GATE_REL, assert_grads_match
from oracle import raster as orc

pytestmark = pytest.mark.gpu

N_MV = 3_000_000
V = 8
GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _region(cam):
    w, h = int(cam["width"]), int(cam["height"])
    x0, y0 = w // 2 - 21, h // 2 - 13  # off the 16-pixel tile grid
    return (x0, y0, x0 + 32, y0 + 32)


@pytest.fixture(scope="module")
def mv_scene():
    g = synth.gaussians(N_MV, 3, seed=1)
    cams = [synth.camera_ring(k, V) for k in range(V)]
    projs = [orc.project(g, c) for c in cams]
    orders = [orc.order(p) for p in projs]
    return g, cams, projs, orders


def _setup(gsp, g, cams):
    import torch
    gs = gsp.GaussianSet.from_arrays(g, capacity=N_MV)
    # a small probe: the pair count is exact even when it exceeds the capacity
    probe = gsp.Renderer(gs, cams, pair_capacity=1 << 20)
    out = probe.forward()
    torch.cuda.synchronize()
    assert int(out["status"].item()) == gsp._lib.GSP_ERR_CAPACITY
    pairs = int(probe.pair_count().item())
    del probe, out
    torch.cuda.empty_cache()
    r = gsp.Renderer(gs, cams, pair_capacity=int(pairs * 1.02) + 4096)
    return gs, r, pairs


def test_3m_eight_uneven_views_graph_autotuned(gsp_lib, mv_scene):
    import torch
    g, cams, projs, orders = mv_scene
    gs, r, pairs = _setup(gsp_lib, g, cams)
    assert pairs > 500_000_000
    gsp_lib.autotune.tune(r)
    offs = r.offsets
    npix = r.total_pix
    # edge map on the regions (zero elsewhere), upstream gradient on the regions
    rng = np.random.default_rng(12)
    e = np.zeros(npix, np.float32)
    dl = np.zeros((npix, 3), np.float32)
    for cam, off in zip(cams, offs):
        w = int(cam["width"])
        x0, y0, x1, y1 = _region(cam)
        for y in range(y0, y1):
            e[off + y * w + x0: off + y * w + x1] = rng.uniform(0.0, 3.0, x1 - x0)
            dl[off + y * w + x0: off + y * w + x1] = rng.normal(size=(x1 - x0, 3)) / npix
    E = torch.from_numpy(e).cuda()
    dL = torch.from_numpy(dl).cuda()
    score = torch.zeros(N_MV, device="cuda")
    grads = {k: torch.zeros_like(getattr(gs, k)) for k in GROUPS}
    bufs = {"rgb": torch.empty((npix, 3), device="cuda"), "T": torch.empty(npix, device="cuda"),
            "last": torch.empty(npix, dtype=torch.int32, device="cuda")}
    status = gsp_lib.new_status()

    def step():
        score.zero_()
        out = r.forward(edge=E, score=score, out=bufs, status=status)
        r.backward(out, dL_drgb=dL, grads=grads, status=status)

    step()  # eager
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    eager = {"rgb": bufs["rgb"].clone(), "score": score.clone(), **{k: v.clone() for k, v in grads.items()}}
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            step()
    torch.cuda.current_stream().wait_stream(side)
    graph.replay()
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert torch.equal(bufs["rgb"], eager["rgb"])  # compositing is deterministic per pixel
    rgb = bufs["rgb"].cpu().numpy()
    T = bufs["T"].cpu().numpy()
    s_gpu = score.cpu().numpy().astype(np.float64)
    grads_all = {k: v.clone() for k, v in grads.items()}
    s_ref = np.zeros(N_MV)
    skip = np.zeros(N_MV, bool)
    per_view, per_mag = [], []
    n_ex = n_px = 0
    for v, (cam, off, proj, order) in enumerate(zip(cams, offs, projs, orders)):
        w, h = int(cam["width"]), int(cam["height"])
        reg = _region(cam)
        x0, y0, x1, y1 = reg
        ev = e[off:off + w * h].reshape(h, w).astype(np.float64)
        ref = orc.render(g, cam, edge=ev, region=reg, proj=proj, order=order)
        ok = ref["gate_gap"][y0:y1, x0:x1] >= GATE_REL
        n_ex += int((~ok).sum())
        n_px += ok.size
        got = rgb[off:off + w * h].reshape(h, w, 3)[y0:y1, x0:x1]
        assert np.abs(got - ref["rgb"][y0:y1, x0:x1]).max(axis=2)[ok].max(initial=0) <= 1e-4
        gotT = T[off:off + w * h].reshape(h, w)[y0:y1, x0:x1]
        assert np.abs(gotT - ref["T"][y0:y1, x0:x1])[ok].max(initial=0) <= 1e-4
        s_ref += ref["score"]
        dlv = dl[off:off + w * h].reshape(h, w, 3).astype(np.float64)
        gr = orc.render_bwd(g, cam, dlv, proj=proj, region=reg)
        per_mag.append(orc.render_bwd(g, cam, dlv, proj=proj, region=reg, magnitude=True))
        if (~ok).any():
            skip |= orc.gate_affected(proj, ref["gate_gap"] < GATE_REL, GATE_REL, order)
        per_view.append(gr)
    assert n_ex <= EXEMPT_FRAC * n_px, (n_ex, n_px)
    floor = 1e-3 * np.abs(s_ref).max()
    rel = np.abs(s_gpu - s_ref) / np.maximum(np.abs(s_ref), floor)
    assert (s_ref > 0).sum() > 500
    assert rel[~skip].max() <= 1e-4, rel[~skip].max()
    # gradients: the batched launch with the upstream gradient on one view at a
    # time against that view's oracle adjoint; then the all-view result against
    # the sum of the per-view results (same FP32 terms, different summation)
    touched = np.zeros(N_MV, bool)
    for gr in per_view:
        touched |= np.abs(gr["opacity_logits"]) > 0
    rows = np.nonzero(touched)[0]
    rows_t = torch.from_numpy(rows).cuda()
    sum_v = {k: 0.0 for k in GROUPS}
    mag_v = {k: 0.0 for k in GROUPS}
    for v, (off, gr, gm) in enumerate(zip(offs, per_view, per_mag)):
        w, h = int(cams[v]["width"]), int(cams[v]["height"])
        dlv = torch.zeros_like(dL)
        dlv[off:off + w * h] = dL[off:off + w * h]
        gv = r.backward(out_keep(r, E, bufs, status), dL_drgb=dlv, status=status)
        torch.cuda.synchronize()
        tv = (np.abs(gr["opacity_logits"]) > 0) & ~skip
        for k in GROUPS:
            a = gv[k][rows_t].cpu().numpy().reshape(rows.size, -1).astype(np.float64)
            b = gr[k][rows].reshape(rows.size, -1)
            m = gm[k][rows].reshape(rows.size, -1)
            kv = tv[rows]
            assert_grads_match(k, a[kv], b[kv], m[kv])
            sum_v[k] = sum_v[k] + a
            mag_v[k] = mag_v[k] + m
    for k in GROUPS:
        a = grads_all[k][rows_t].cpu().numpy().reshape(rows.size, -1).astype(np.float64)
        assert_grads_match(k, a, sum_v[k], mag_v[k])
        mask = torch.ones(N_MV, dtype=torch.bool, device="cuda")
        mask[rows_t] = False
        assert bool((grads_all[k][mask] == 0).all())


def out_keep(r, E, bufs, status):
    """The forward outputs of the last forward pass (buffers kept by the caller)."""
    return {"rgb": bufs["rgb"], "T": bufs["T"], "last": bufs["last"], "loss": None, "status": status}


def test_compositing_variants_agree(gsp_lib):
    import torch
    g = synth.gaussians(20000, 3, seed=6)
    cams = [synth.camera_ring(k, 3, resolutions=[(320, 240), (257, 193), (400, 300)]) for k in range(3)]
    gs = gsp_lib.GaussianSet.from_arrays(g)
    r = gsp_lib.Renderer(gs, cams, pair_capacity=1 << 24)
    rng = np.random.default_rng(1)
    E = torch.from_numpy(rng.uniform(0, 2, r.total_pix).astype(np.float32)).cuda()
    dL = torch.from_numpy(rng.normal(size=(r.total_pix, 3)).astype(np.float32) / r.total_pix).cuda()
    res = []
    for fv in range(gsp_lib._lib.GSP_FWD_VARIANTS):
        r.variants = (fv, 0)
        sc = torch.zeros(gs.capacity, device="cuda")
        out = r.forward(edge=E, score=sc)
        res.append((out["rgb"].clone(), out["T"].clone(), out["last"].clone(), sc))
    for a in res[1:]:
        assert torch.equal(a[0], res[0][0]) and torch.equal(a[1], res[0][1]) and torch.equal(a[2], res[0][2])
        torch.testing.assert_close(a[3], res[0][3], rtol=1e-5, atol=1e-6)
    grads = []
    for bv in range(gsp_lib._lib.GSP_BWD_VARIANTS):
        r.variants = (0, bv)
        out = r.forward()
        grads.append(r.backward(out, dL_drgb=dL))
    torch.cuda.synchronize()
    for gr in grads[1:]:
        for k in GROUPS:
            torch.testing.assert_close(gr[k], grads[0][k], rtol=1e-4, atol=1e-9)
