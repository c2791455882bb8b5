"""The bounds-checked build (libgsp_debug.so, compiled with -DGSP_DEBUG) runs
the whole step at full size with no index out of bounds, and computes what
the release build computes.

Each build runs in its own process (GSP_LIBRARY names the library the
package loads): one step of 1,000,000 SH-3 Gaussians over four ring views of
1237x822 - edge map (tile kernel), batched forward with L1 loss and edge
score, adjoint, top 10 % selection, Long-Axis-Split - and then a 32-view
1237x822 edge map (walk kernel).  Every status word of the bounds-checked run
must be 0 (an index out of bounds records GSP_ERR_CAPACITY and skips the
access).  Its results must equal the release run's: bitwise for everything
computed without floating-point atomics (edge maps, medians, rendered RGB and
T, the selection mask and the split Gaussians, both given the release run's
scores); the loss, scores and gradients, summed by atomics in an order that
changes from run to run, within 1e-5 of their group's 2-norm and 1e-4 of its
largest entry.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2603_08661_gb300")
N, W, H, VIEWS = 1_000_000, 1237, 822, 4
CAP = N + N // 10
GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def run_step(outdir: str, tag: str, ref_scores: str | None) -> None:
    """One full-size step with the library the environment names; results to
    outdir/<tag>.npz.  ref_scores: a .npy of scores to select from (the
    release run's), else the step's own."""
    sys.path.insert(0, ROOT)
    import torch

    import paper_2603_08661_gb300 as gsp
    import synth
    res = {}
    stat = {}
    g = synth.gaussians(N, 3, seed=1)
    cams = [synth.camera_ring(k, VIEWS, resolutions=[(W, H)]) for k in range(VIEWS)]
    targets = [torch.from_numpy(synth.image(H, W, 3000 + k)).cuda() for k in range(VIEWS)]
    E, med, _, st = gsp.edge_map(targets)
    stat["edge"] = st
    gs = gsp.GaussianSet.from_arrays(g, capacity=CAP)
    probe = gsp.Renderer(gs, cams, pair_capacity=1 << 28)
    probe.forward()
    torch.cuda.synchronize()
    pairs = int(probe.pair_count().item())
    del probe
    r = gsp.Renderer(gs, cams, pair_capacity=int(pairs * 1.05) + 1024)
    score = torch.zeros(CAP, device="cuda")
    fwd = r.forward(targets=targets, edge=E, score=score)
    grads = r.backward(fwd, targets=targets)
    stat["render"] = fwd["status"]
    sc = torch.from_numpy(np.load(ref_scores)).cuda() if ref_scores else score
    mask, sel, st = gsp.topk_mask(sc, gs.count, N // 10)
    stat["topk"] = st
    stat["las"] = gsp.las_split(gs, mask=mask)
    imgs32 = [torch.from_numpy(synth.image(H, W, 4000 + k)).cuda() for k in range(32)]
    E32, med32, _, st = gsp.edge_map(imgs32)
    stat["edge32"] = st
    torch.cuda.synchronize()
    res.update(E=E, med=med, rgb=fwd["rgb"], T=fwd["T"], loss=fwd["loss"], score=score, mask=mask,
               count=gs.count, E32=E32, med32=med32)
    for k in GROUPS:
        res["grad_" + k] = grads[k]
        res["split_" + k] = getattr(gs, k)
    out = {k: v.cpu().numpy() for k, v in res.items()}
    out.update({"status_" + k: np.int64(v.item()) for k, v in stat.items()})
    np.savez(os.path.join(outdir, tag + ".npz"), **out)


def _spawn(outdir, tag, library, ref_scores=None):
    env = dict(os.environ, GSP_LIBRARY=library)
    code = ("import sys; sys.path[:0] = [%r, %r]; import test_gpu_debug_bounds as t; t.run_step(%r, %r, %r)"
            % (ROOT, os.path.dirname(os.path.abspath(__file__)), str(outdir), tag, ref_scores))
    p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stderr[-3000:]
    return np.load(os.path.join(outdir, tag + ".npz"))


def _close(a, b, name):
    a = a.astype(np.float64).ravel()
    b = b.astype(np.float64).ravel()
    d = np.abs(a - b)
    assert np.sqrt((d ** 2).sum()) <= 1e-5 * np.sqrt((b ** 2).sum()) + 1e-30, name
    assert d.max(initial=0) <= 1e-4 * np.abs(b).max(initial=0) + 1e-30, name


def test_bounds_checked_build_runs_clean_and_matches_release(gsp_lib, tmp_path):
    debug_lib = os.path.join(PKG, "libgsp_debug.so")
    assert os.path.exists(debug_lib), "libgsp_debug.so is built by __graft_entry__.build()"
    rel = _spawn(tmp_path, "release", os.path.join(PKG, "libgsp.so"))
    np.save(tmp_path / "scores.npy", rel["score"])
    dbg = _spawn(tmp_path, "debug", debug_lib, str(tmp_path / "scores.npy"))
    for k in ("edge", "render", "topk", "las", "edge32"):
        assert int(rel["status_" + k]) == 0, k
        assert int(dbg["status_" + k]) == 0, k
    for k in ("E", "med", "rgb", "T", "mask", "count", "E32", "med32"):
        assert np.array_equal(dbg[k], rel[k]), k
    assert int(rel["mask"].sum()) == N // 10 and int(rel["count"][0]) == N + N // 10
    for k in GROUPS:
        assert np.array_equal(dbg["split_" + k], rel["split_" + k]), k
        _close(dbg["grad_" + k], rel["grad_" + k], k)
    _close(dbg["score"], rel["score"], "score")
    _close(dbg["loss"], rel["loss"], "loss")
