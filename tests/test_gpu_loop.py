"""The device-resident densification loop, scaled down: 4 views, 4,000 -> 6,000
Gaussians in 4 events of 500 every 5 iterations, SGD with lr 1e-3.

* The first iteration's gradients (L1 loss over all pixels of the 4 views)
  match the oracle's analytic adjoint entry by entry (sums over views:
  conftest.grad_bound), and the SGD step is one FMA per element.
* A densification event equals the oracle's top-k on the accumulated scores
  (exact) and its Long-Axis-Split of the pre-event state (1e-6).
* The CUDA-graph driver and the autograd driver agree on an iteration, and
  the graph driver reaches the budget with the count on the device.
"""
import numpy as np
import pytest

import synth
from conftest import assert_grads_match
from oracle import densify as od
from oracle import raster as orc

pytestmark = pytest.mark.gpu

N0, CAP, K_EVENT, EVERY, LR = 4000, 6000, 500, 5, 1e-3
W, H, V = 96, 64, 4
GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _make(gsp):
    import torch
    g = synth.gaussians(N0, 3, seed=11)
    g["log_scales"] = (g["log_scales"] + 0.8).astype(np.float32)
    cams = [synth.camera_ring(k, V, resolutions=[(W, H)]) for k in range(V)]
    tg = [synth.image(H, W, 2000 + k) for k in range(V)]
    gs = gsp.GaussianSet.from_arrays(g, capacity=CAP)
    loop = gsp.DensifyLoop(gs, cams, [torch.from_numpy(t).cuda() for t in tg], lr=LR, every=EVERY,
                           k_event=K_EVENT, pair_capacity=1 << 22, las=gsp.LAS_CONFIG)
    return g, cams, tg, gs, loop


def _host(gs, n):
    return {k: getattr(gs, k)[:n].cpu().numpy().astype(np.float64) for k in GROUPS}


def test_first_iteration_gradients_and_sgd_step(gsp_lib):
    import torch
    g, cams, tg, gs, loop = _make(gsp_lib)
    p0 = {k: getattr(gs, k)[:N0].cpu().numpy() for k in GROUPS}
    loop.iteration()
    torch.cuda.synchronize()
    assert int(loop.status.item()) == 0
    p1 = {k: getattr(gs, k)[:N0].cpu().numpy() for k in GROUPS}
    gg = {k: loop.grads[k][:N0].cpu().numpy() for k in GROUPS}
    # SGD: one FMA per element, fma(-lr, grad, theta) rounded once to FP32
    for k in GROUPS:
        ref = (p0[k].astype(np.float64) + np.float64(np.float32(-LR)) * gg[k].astype(np.float64)).astype(np.float32)
        ulp = np.spacing(np.abs(ref))
        assert np.all(np.abs(p1[k].astype(np.float64) - ref) <= ulp)
    # gradients of the L1 loss (mean over all pixels of all views) against the oracle
    total = V * W * H
    ref_g = {k: 0.0 for k in GROUPS}
    mag_g = {k: 0.0 for k in GROUPS}
    for cam, t in zip(cams, tg):
        out = orc.render(g, cam)
        diff = out["rgb"] - t / 255.0
        assert ((np.abs(diff) < 1e-5) & (diff != 0)).sum() == 0  # no L1 sign is a near-tie
        dl = np.sign(diff) / (3.0 * total)
        gr = orc.render_bwd(g, cam, dl, proj=out["proj"])
        gm = orc.render_bwd(g, cam, dl, proj=out["proj"], magnitude=True)
        for k in GROUPS:
            ref_g[k] = ref_g[k] + gr[k].reshape(N0, -1)
            mag_g[k] = mag_g[k] + gm[k].reshape(N0, -1)
    for k in GROUPS:
        a = gg[k].reshape(N0, -1).astype(np.float64)
        assert_grads_match(k, a, ref_g[k], mag_g[k])


def test_event_matches_oracle_topk_and_split(gsp_lib):
    import torch
    g, cams, tg, gs, loop = _make(gsp_lib)
    for _ in range(EVERY):
        loop.iteration()
    torch.cuda.synchronize()
    before = _host(gs, N0)
    before["sh_degree"] = 3
    scores = loop.score[:N0].cpu().numpy()
    loop.event()
    torch.cuda.synchronize()
    assert int(loop.status.item()) == 0 and int(gs.count.item()) == N0 + K_EVENT
    mask = loop.mask[:N0].cpu().numpy().astype(bool)
    assert np.array_equal(mask, od.topk_mask(scores.astype(np.float64), K_EVENT))
    p32 = {k: float(np.float32(v)) for k, v in od.CONFIG_PRESET.items()}
    ref = od.las_split(before, mask, **p32)
    for k in GROUPS:
        got = getattr(gs, k)[:N0 + K_EVENT].cpu().numpy().astype(np.float64).reshape(N0 + K_EVENT, -1)
        want = ref[k].reshape(N0 + K_EVENT, -1)
        assert (np.abs(got - want) / np.maximum(1.0, np.abs(want))).max() <= 1e-6, k
    assert float(loop.score.abs().max().item()) == 0.0


def test_graph_driver_reaches_budget_and_agrees_with_autograd(gsp_lib):
    import torch
    _, _, _, gs_a, loop_a = _make(gsp_lib)
    _, _, _, gs_b, loop_b = _make(gsp_lib)
    la = loop_a.step_autograd()
    loop_b.run(1)
    torch.cuda.synchronize()
    assert abs(float(la.item()) - float(loop_b.loss().item())) <= 1e-6 * float(la.item())
    for k in GROUPS:
        torch.testing.assert_close(getattr(gs_a, k), getattr(gs_b, k), rtol=1e-6, atol=1e-9)
    losses = [float(loop_b.loss().item())]
    for _ in range(4 * EVERY - 1):
        loop_b.run(1)
        losses.append(float(loop_b.loss().item()))
    torch.cuda.synchronize()
    assert int(loop_b.status.item()) == 0
    assert int(gs_b.count.item()) == N0 + 4 * K_EVENT == CAP
    assert np.all(np.isfinite(losses))
    assert all(torch.isfinite(getattr(gs_b, k)).all() for k in GROUPS)


def test_gated_event_after_warmup_matches_oracle(gsp_lib):
    """Gradient-threshold masking in the loop: the first event (warm-up) selects
    by score alone and clears the statistic; the next one selects the top-k among
    the candidates of the statistic accumulated since, exactly as the oracle does
    on the same score and statistic arrays.  The graph driver then replays both
    kinds of event."""
    import torch
    g = synth.gaussians(N0, 3, seed=11)
    g["log_scales"] = (g["log_scales"] + 0.8).astype(np.float32)
    cams = [synth.camera_ring(k, V, resolutions=[(W, H)]) for k in range(V)]
    tg = [torch.from_numpy(synth.image(H, W, 2000 + k)).cuda() for k in range(V)]
    gs = gsp_lib.GaussianSet.from_arrays(g, capacity=CAP + 2 * K_EVENT)
    loop = gsp_lib.DensifyLoop(gs, cams, tg, lr=LR, every=EVERY, k_event=K_EVENT, pair_capacity=1 << 22,
                               grad_threshold=0.0, warmup_events=1)
    for _ in range(EVERY):
        loop.iteration()
    assert not loop.gated()
    loop.event()
    torch.cuda.synchronize()
    assert int(loop.status.item()) == 0 and loop.events == 1 and loop.gated()
    assert int(loop.pos_grad[1].sum().item()) == 0 and float(loop.pos_grad[0].abs().sum().item()) == 0.0
    n1 = int(gs.count.item())
    assert n1 == N0 + K_EVENT
    for _ in range(EVERY):
        loop.iteration()
    torch.cuda.synchronize()
    sums = loop.pos_grad[0][:n1].cpu().numpy()
    cnts = loop.pos_grad[1][:n1].cpu().numpy()
    score = loop.score[:n1].cpu().numpy()
    seen = cnts > 0
    assert seen.sum() > n1 // 4
    mean = sums[seen] / cnts[seen]
    loop.grad_threshold = float(np.median(mean))  # about half the seen Gaussians pass
    ref = od.gated_topk_mask(score, K_EVENT, sums, cnts, loop.grad_threshold)
    assert 0 < ref.sum() <= K_EVENT
    loop.event()
    torch.cuda.synchronize()
    assert int(loop.status.item()) == 0
    m = loop.mask[:n1].cpu().numpy().astype(bool)
    assert np.array_equal(m, ref)
    assert int(gs.count.item()) == n1 + int(ref.sum()) == n1 + int(loop.selected.item())
    # graph driver: two more events, both gated
    loop.run(2 * EVERY)
    torch.cuda.synchronize()
    assert int(loop.status.item()) == 0 and loop.events == 4
    assert int(gs.count.item()) <= CAP + 2 * K_EVENT


def test_sampling_event_matches_oracle_and_paper_preset_is_default(gsp_lib):
    """selection = "sample": the event draws fresh Exp(1) variates and samples k
    Gaussians by score; the mask equals the oracle's exponential-clock sample for
    the same scores and variates, and the split uses the paper's LAS preset."""
    import torch
    g = synth.gaussians(N0, 3, seed=11)
    g["log_scales"] = (g["log_scales"] + 0.8).astype(np.float32)
    cams = [synth.camera_ring(k, V, resolutions=[(W, H)]) for k in range(V)]
    tg = [torch.from_numpy(synth.image(H, W, 2000 + k)).cuda() for k in range(V)]
    gs = gsp_lib.GaussianSet.from_arrays(g, capacity=CAP)
    loop = gsp_lib.DensifyLoop(gs, cams, tg, lr=LR, every=EVERY, k_event=K_EVENT, pair_capacity=1 << 22,
                               selection="sample")
    for _ in range(EVERY):
        loop.iteration()
    torch.cuda.synchronize()
    score = loop.score[:N0].cpu().numpy()
    before = _host(gs, N0)
    before["sh_degree"] = 3
    loop.event()
    torch.cuda.synchronize()
    assert int(loop.status.item()) == 0
    ref = od.sample_mask(score, loop.expv[:N0].cpu().numpy(), K_EVENT)
    m = loop.mask[:N0].cpu().numpy().astype(bool)
    assert np.array_equal(m, ref) and ref.sum() == min(K_EVENT, int((score > 0).sum()))
    n1 = int(gs.count.item())
    assert n1 == N0 + int(ref.sum())
    p32 = {k: float(np.float32(v)) for k, v in od.PAPER_PRESET.items()}
    split = od.las_split(before, ref, **p32)
    after = _host(gs, n1)
    for k in ("means", "log_scales", "opacity_logits"):
        a, b = after[k].reshape(n1, -1), split[k].reshape(n1, -1)
        assert (np.abs(a - b) / np.maximum(1.0, np.abs(b))).max() <= 1e-6, k


def test_schedule_window_and_budget_in_the_graph_driver(gsp_lib):
    """The paper's refinement set-up scaled down: events every EVERY iterations only
    inside [2 EVERY, 4 EVERY], the Gaussian count never above the budget (the last
    event is cut to the room left), the learning rates decaying on the device (the
    step counter advances once per iteration, graph replays included)."""
    import torch
    g = synth.gaussians(N0, 3, seed=11)
    g["log_scales"] = (g["log_scales"] + 0.8).astype(np.float32)
    cams = [synth.camera_ring(k, V, resolutions=[(W, H)]) for k in range(V)]
    tg = [torch.from_numpy(synth.image(H, W, 2000 + k)).cuda() for k in range(V)]
    budget = N0 + 2 * K_EVENT + 123
    gs = gsp_lib.GaussianSet.from_arrays(g, capacity=CAP)
    sched = {"steps": 30, "means": (1.28e-4, 1.28e-5), "log_scales": (0.020, 0.002)}
    loop = gsp_lib.DensifyLoop(gs, cams, tg, lr=LR, every=EVERY, k_event=K_EVENT, pair_capacity=1 << 22,
                               schedule=sched, densify_from=2 * EVERY, densify_until=4 * EVERY, budget=budget)
    counts = []
    for it in range(6):  # 6 x EVERY iterations, one replay block at a time
        loop.run(EVERY)
        torch.cuda.synchronize()
        assert int(loop.status.item()) == 0
        counts.append(int(gs.count.item()))
    assert loop.events == 3  # iterations 2 EVERY, 3 EVERY, 4 EVERY
    assert counts == [N0, N0 + K_EVENT, N0 + 2 * K_EVENT, budget, budget, budget]
    assert int(loop.step_dev.item()) == 6 * EVERY
