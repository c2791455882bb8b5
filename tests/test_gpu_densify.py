"""GPU top-k selection and Long-Axis-Split (Sec. 2.2, Alg. 1-2) against the oracle.

Selection is integer work: masks must match exactly for the same scores.
LAS parameters match within 1e-6 (max of absolute and relative) given the
same selection.
"""
import numpy as np
import pytest

import synth
from oracle import densify as od

pytestmark = pytest.mark.gpu


def _las_close(got, ref, tol=1e-6):
    err = np.abs(got - ref) / np.maximum(1.0, np.abs(ref))
    assert err.max(initial=0) <= tol, err.max()


@pytest.mark.parametrize("n,k", [(1, 0), (1, 1), (7, 3), (1000, 100), (4097, 4097), (300000, 30000)])
def test_topk_matches_oracle_with_ties(gsp_lib, n, k):
    import torch
    rng = np.random.default_rng(n + k)
    s = rng.integers(0, 50, n).astype(np.float32) * np.float32(0.25)  # many ties
    s[rng.integers(0, n, max(n // 10, 1))] = -rng.uniform(0, 3, max(n // 10, 1)).astype(np.float32)
    cap = n + 5
    sc = torch.zeros(cap, device="cuda")
    sc[:n] = torch.from_numpy(s).cuda()
    cnt = torch.tensor([n], dtype=torch.int32, device="cuda")
    mask, sel, st = gsp_lib.topk_mask(sc, cnt, k)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    m = mask.cpu().numpy().astype(bool)
    assert not m[n:].any()
    assert np.array_equal(m[:n], od.topk_mask(s, k))
    assert int(sel.item()) == k


def test_topk_continuous_scores_and_k_beyond_n(gsp_lib):
    import torch
    s = np.random.default_rng(0).gamma(2.0, 1.0, 50000).astype(np.float32)
    sc = torch.from_numpy(s).cuda()
    cnt = torch.tensor([50000], dtype=torch.int32, device="cuda")
    for k in (0, 1, 4999, 50000, 70000):
        mask, sel, _ = gsp_lib.topk_mask(sc, cnt, k)
        m = mask.cpu().numpy().astype(bool)
        assert np.array_equal(m, od.topk_mask(s, min(k, 50000)))


@pytest.mark.parametrize("preset", ["config", "paper"])
@pytest.mark.parametrize("sh_degree", [0, 3])
def test_las_matches_oracle(gsp_lib, preset, sh_degree):
    import torch
    n = 5000
    g = synth.gaussians(n, sh_degree, seed=21)
    g["quats"] = (g["quats"] * np.random.default_rng(2).uniform(0.5, 2, (n, 1))).astype(np.float32)
    mask = np.zeros(n, bool)
    mask[np.random.default_rng(3).choice(n, 700, replace=False)] = True
    params = gsp_lib.LAS_CONFIG if preset == "config" else gsp_lib.LAS_PAPER
    gs = gsp_lib.GaussianSet.from_arrays(g, capacity=n + 1000)
    st = gsp_lib.las_split(gs, mask=torch.from_numpy(mask.astype(np.uint8)).cuda(), params=params)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and int(gs.count.item()) == n + 700
    p32 = {k: float(np.float32(v)) for k, v in params.items()}
    ref = od.las_split(g, mask, **p32)
    for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        got = getattr(gs, name)[:n + 700].cpu().numpy().astype(np.float64)
        _las_close(got.reshape(n + 700, -1), ref[name].reshape(n + 700, -1))


def test_las_capacity_overflow_changes_nothing(gsp_lib):
    import torch
    n = 1000
    g = synth.gaussians(n, 1, seed=5)
    gs = gsp_lib.GaussianSet.from_arrays(g, capacity=n + 10)
    before = {k: getattr(gs, k).clone() for k in ("means", "log_scales", "opacity_logits")}
    mask = torch.ones(n + 10, dtype=torch.uint8, device="cuda")
    st = gsp_lib.las_split(gs, mask=mask)
    torch.cuda.synchronize()
    assert int(st.item()) == gsp_lib._lib.GSP_ERR_CAPACITY
    assert int(gs.count.item()) == n
    for k, v in before.items():
        assert torch.equal(getattr(gs, k), v)


def test_las_topk_path_equals_mask_path(gsp_lib):
    import torch
    n = 20000
    g = synth.gaussians(n, 3, seed=9)
    scores = torch.from_numpy(np.random.default_rng(1).gamma(2, 1, n).astype(np.float32)).cuda()
    a = gsp_lib.GaussianSet.from_arrays(g, capacity=n + 3000)
    b = gsp_lib.GaussianSet.from_arrays(g, capacity=n + 3000)
    sc = torch.zeros(n + 3000, device="cuda")
    sc[:n] = scores
    gsp_lib.las_split(a, scores=sc, k=2000)
    mask, _, _ = gsp_lib.topk_mask(sc, b.count, 2000)
    gsp_lib.las_split(b, mask=mask)
    torch.cuda.synchronize()
    for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        assert torch.equal(getattr(a, name), getattr(b, name))
    assert int(a.count.item()) == n + 2000


def test_config0_pipeline_selection_and_split(gsp_lib):
    """Edge map -> render with score -> top 10% -> LAS on the tiny configuration."""
    import torch
    from oracle import edge as oe
    from oracle import raster as orc
    g = synth.gaussians(2000, 0, seed=1)
    cam = synth.camera_front(128, 128)
    tgt = synth.image(128, 128, 2000)
    t = torch.from_numpy(tgt).cuda()
    E, med, _, _ = gsp_lib.edge_map([t])
    gs = gsp_lib.GaussianSet.from_arrays(g, capacity=2200)
    r = gsp_lib.Renderer(gs, [cam], 1 << 20)
    score = torch.zeros(2200, device="cuda")
    r.forward(targets=[t], edge=E, score=score)
    mask, sel, st = gsp_lib.topk_mask(score, gs.count, 200)
    gsp_lib.las_split(gs, mask=mask, status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and int(gs.count.item()) == 2200
    ref_e = oe.edge_map(tgt)["E"]
    ref = orc.render(g, cam, edge=ref_e)
    m = mask.cpu().numpy().astype(bool)[:2000]
    ref_m = od.topk_mask(ref["score"], 200)
    kth = np.sort(ref["score"])[::-1][199]
    near = np.abs(ref["score"] - kth) <= 1e-4 * kth
    assert ((m != ref_m) & ~near).sum() == 0
    ref_las = od.las_split(g, m, **od.CONFIG_PRESET)
    _las_close(gs.means[:2200].cpu().numpy().astype(np.float64), ref_las["means"])


def _gate_inputs(n, seed):
    rng = np.random.default_rng(seed)
    s = rng.integers(0, 40, n).astype(np.float32) * np.float32(0.5)  # ties
    cnt = rng.integers(0, 5, n).astype(np.int32)  # count 0: never seen
    sums = (rng.gamma(2.0, 1e-4, n) * cnt).astype(np.float32)
    return s, sums, cnt


@pytest.mark.parametrize("n,k,tau", [(1, 1, 0.0), (9, 4, 1e-4), (5000, 600, 2e-4), (5000, 5000, 1e-4),
                                     (300000, 30000, 2.5e-4), (1000000, 100000, 1.5e-4)])
def test_gated_topk_matches_oracle(gsp_lib, n, k, tau):
    """Gradient-threshold masking fused into the selection: bit-exact masks and
    counts, candidate decision in FP32 on both sides; k may exceed the candidates."""
    import torch
    s, sums, cnt = _gate_inputs(n, n + k)
    cap = n + 3
    dev = lambda a, dt: torch.from_numpy(np.concatenate([a, np.zeros(3, a.dtype)])).to("cuda", dt)
    cnt_t = torch.tensor([n], dtype=torch.int32, device="cuda")
    mask, sel, st = gsp_lib.topk_mask_gated(dev(s, torch.float32), dev(sums, torch.float32),
                                            dev(cnt, torch.int32), tau, cnt_t, k)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    m = mask.cpu().numpy().astype(bool)
    ref = od.gated_topk_mask(s, k, sums, cnt, tau)
    assert not m[n:].any()
    assert np.array_equal(m[:n], ref)
    assert int(sel.item()) == int(ref.sum()) == min(k, int(od.grad_candidates(sums, cnt, tau).sum()))


def test_gated_topk_limits(gsp_lib):
    import torch
    s, sums, cnt = _gate_inputs(20000, 5)
    t = lambda a: torch.from_numpy(a).cuda()
    n_t = torch.tensor([20000], dtype=torch.int32, device="cuda")
    # infinite threshold: nothing; threshold 0 with every count > 0: plain top-k
    mask, sel, _ = gsp_lib.topk_mask_gated(t(s), t(sums), t(cnt), float("inf"), n_t, 500)
    assert int(sel.item()) == 0 and not mask.any()
    ones = np.maximum(cnt, 1).astype(np.int32)
    mask, _, _ = gsp_lib.topk_mask_gated(t(s), t(sums), t(ones), 0.0, n_t, 500)
    plain, _, _ = gsp_lib.topk_mask(t(s), n_t, 500)
    assert torch.equal(mask, plain)
    with pytest.raises(Exception):
        gsp_lib.topk_mask_gated(t(s), t(sums), t(cnt), float("nan"), n_t, 500)


@pytest.mark.parametrize("n,k", [(1, 1), (50, 10), (5000, 700), (5000, 9000), (1000000, 100000)])
def test_importance_sampling_matches_oracle(gsp_lib, n, k):
    """Exponential-clock sampling by score: bit-exact masks for the same scores and
    Exp(1) variates (ringing times are one FP32 division on both sides), with
    non-positive scores, equal scores and repeated variates (tied times)."""
    import torch
    rng = np.random.default_rng(n * 7 + k)
    s = rng.gamma(1.5, 1.0, n).astype(np.float32)
    s[rng.integers(0, n, max(n // 20, 1))] = 0.0
    s[rng.integers(0, n, max(n // 50, 1))] = -1.0
    s[rng.integers(0, n, max(n // 10, 1))] = np.float32(2.0)
    e = rng.exponential(size=n).astype(np.float32)
    e[rng.integers(0, n, max(n // 10, 1))] = np.float32(0.5)
    cap = n + 2
    pad = lambda a: torch.from_numpy(np.concatenate([a, np.ones(2, np.float32)])).cuda()
    cnt = torch.tensor([n], dtype=torch.int32, device="cuda")
    mask, sel, st = gsp_lib.sample_mask(pad(s), pad(e), cnt, k)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    m = mask.cpu().numpy().astype(bool)
    ref = od.sample_mask(s, e, k)
    assert not m[n:].any()
    assert np.array_equal(m[:n], ref)
    assert int(sel.item()) == int(ref.sum()) == min(k, int((s > 0).sum()))


@pytest.mark.parametrize("mode", ["topk", "gated", "sample"])
@pytest.mark.parametrize("budget", [0, 20300, 20000, 19000])
def test_select_mask_budget(gsp_lib, mode, budget):
    """gsp_select_mask: the selection of each mode with k reduced to the room left
    under the budget (at most budget - N selected; none when N >= budget)."""
    import torch
    n, k = 20000, 1000
    s, sums, cnt = _gate_inputs(n, 77)
    e = np.random.default_rng(78).exponential(size=n).astype(np.float32)
    t = lambda a: torch.from_numpy(a).cuda()
    n_t = torch.tensor([n], dtype=torch.int32, device="cuda")
    kb = od.budgeted_k(k, n, budget)
    tau = 2e-4
    if mode == "topk":
        mask, sel, st = gsp_lib.select_mask(t(s), n_t, k, budget=budget)
        ref = od.topk_mask(s, kb)
    elif mode == "gated":
        mask, sel, st = gsp_lib.select_mask(t(s), n_t, k, pos_grad=(t(sums), t(cnt)), threshold=tau, budget=budget)
        ref = od.gated_topk_mask(s, kb, sums, cnt, tau)
    else:
        mask, sel, st = gsp_lib.select_mask(t(s), n_t, k, exp_variates=t(e), budget=budget)
        ref = od.sample_mask(s, e, kb)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert np.array_equal(mask.cpu().numpy().astype(bool), ref)
    assert int(sel.item()) == int(ref.sum()) <= kb


def test_scheduled_sgd_follows_the_oracle_schedule(gsp_lib):
    """gsp_sgd_step_scheduled: every step uses each group's rate at the device step
    (the paper's decays for means and log-scales over 4 steps, constant rates for the
    rest), then advances the step; held at lr_final after the horizon."""
    import ctypes
    import torch
    from oracle import optim as oo
    from paper_2603_08661_gb300 import _lib as L
    n, steps = 3000, 4
    g = synth.gaussians(n, 3, seed=5)
    gs = gsp_lib.GaussianSet.from_arrays(g)
    rng = np.random.default_rng(6)
    grads = {k: torch.from_numpy(rng.normal(size=getattr(gs, k).shape).astype(np.float32)).cuda()
             for k in oo.GROUPS}
    rates = {"means": oo.PAPER_SCHEDULE["means"], "log_scales": oo.PAPER_SCHEDULE["log_scales"],
             "quats": (1e-3, 1e-3), "opacity_logits": (5e-2, 5e-2), "sh": (2.5e-3, 2.5e-3)}
    sched = L.LrSchedule((L.c_f32 * 5)(*[rates[k][0] for k in oo.GROUPS]),
                         (L.c_f32 * 5)(*[rates[k][1] for k in oo.GROUPS]), steps)
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    for t in range(steps + 2):
        before = {k: getattr(gs, k).cpu().numpy().astype(np.float64) for k in oo.GROUPS}
        L.check(gsp_lib._lib.load().gsp_sgd_step_scheduled(ctypes.byref(gs.struct()),
                                                            *[gsp_lib.api._ptr(grads[k]) for k in oo.GROUPS],
                                                            ctypes.byref(sched), gsp_lib.api._ptr(step), None), "sgd")
        torch.cuda.synchronize()
        assert int(step.item()) == t + 1
        for k in oo.GROUPS:
            lr = oo.lr_at(rates[k][0], rates[k][1], steps, t)
            gk = grads[k].cpu().numpy().astype(np.float64)
            ref = before[k] - lr * gk
            got = getattr(gs, k).cpu().numpy().astype(np.float64)
            # FP32 rate (1e-6 relative) times the gradient, plus one rounding of theta
            tol = 2e-6 * lr * np.abs(gk) + np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
            assert np.all(np.abs(got - ref) <= tol), (k, t)


def test_selection_started_from_the_score_event(gsp_lib):
    """gsp_render_bwd records the score event once the edge score is complete: a
    selection started from it on a second stream, while the adjoint still chains
    the gradients to the parameters, equals the oracle's top-k of the final
    scores."""
    import torch
    n, k = 60000, 6000
    g = synth.gaussians(n, 3, seed=31)
    cam = synth.camera_front(320, 240)
    t = torch.from_numpy(synth.image(240, 320, 77)).cuda()
    E, _, _, _ = gsp_lib.edge_map([t])
    gs = gsp_lib.GaussianSet.from_arrays(g)
    r = gsp_lib.Renderer(gs, [cam], pair_capacity=1 << 24)
    score = torch.zeros(n, device="cuda")
    ev = torch.cuda.Event()
    side = torch.cuda.Stream()
    out = r.forward(targets=[t])
    r.backward(out, targets=[t], edge=E, score=score, score_event=ev)
    side.wait_event(ev)
    with torch.cuda.stream(side):
        mask, sel, st = gsp_lib.select_mask(score, gs.count, k)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    assert int(out["status"].item()) == 0 and int(st.item()) == 0
    s = score.cpu().numpy()
    assert (s > 0).sum() > k
    assert np.array_equal(mask.cpu().numpy().astype(bool), od.topk_mask(s.astype(np.float64), k))
    assert int(sel.item()) == k
