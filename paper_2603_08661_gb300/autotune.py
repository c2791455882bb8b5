"""Autotuner for the compositing variants of a workload.

gsp_render_fwd / gsp_render_bwd each have a few kernel variants (pixels per
thread, Gaussians staged per shared-memory batch; include/gsp.h lists them).
They give the same results and differ only in speed, which depends on the
scene, the views and the GPU.  `tune` times every variant of each pass on the
caller's renderer with CUDA events and keeps the fastest; choices are cached
per workload signature (GPU, capacity, SH degree, view sizes, pair capacity)
in memory and, when a path is given, in a JSON file.
"""
from __future__ import annotations

import json
import os

import torch

from . import _lib as L


def signature(renderer) -> str:
    dev = torch.cuda.get_device_name(renderer.device)
    views = ",".join(f"{c.width}x{c.height}" for c in renderer.cams)
    return f"{dev}|cap={renderer.gs.capacity}|sh={renderer.gs.sh_degree}|views={views}|pairs={renderer.opts.pair_capacity}"


_cache: dict[str, tuple[int, int]] = {}


def _time(fn, reps: int) -> float:
    fn()  # warm-up (also instantiates the module's kernels)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def tune(renderer, targets=None, dL_drgb=None, reps: int = 3, cache_path: str | None = None,
         verbose: bool = False) -> tuple[int, int]:
    """Pick the fastest forward and adjoint variants for this renderer's workload
    and set them on the renderer.  The adjoint is timed with the L1 loss of
    targets, else with dL_drgb, else with a constant upstream gradient.
    Returns (fwd_variant, bwd_variant)."""
    key = signature(renderer)
    if cache_path and os.path.exists(cache_path) and key not in _cache:
        try:
            _cache.update({k: tuple(v) for k, v in json.load(open(cache_path)).items()})
        except (OSError, ValueError):
            pass
    if key in _cache:
        renderer.variants = _cache[key]
        return _cache[key]
    saved = renderer.variants
    timings_f, timings_b = [], []
    for fv in range(L.GSP_FWD_VARIANTS):
        renderer.variants = (fv, saved[1])
        timings_f.append(_time(lambda: renderer.forward(targets=targets), reps))
    best_f = min(range(len(timings_f)), key=timings_f.__getitem__)
    renderer.variants = (best_f, saved[1])
    out = renderer.forward(targets=targets)
    if targets is None and dL_drgb is None:
        dL_drgb = torch.full((renderer.total_pix, 3), 1.0 / renderer.total_pix, device=renderer.device)
    grads = None
    for bv in range(L.GSP_BWD_VARIANTS):
        renderer.variants = (best_f, bv)

        def bwd():
            nonlocal grads
            grads = renderer.backward(out, targets=targets if dL_drgb is None else None, dL_drgb=dL_drgb,
                                      grads=grads)

        timings_b.append(_time(bwd, reps))
    best_b = min(range(len(timings_b)), key=timings_b.__getitem__)
    choice = (best_f, best_b)
    renderer.variants = choice
    _cache[key] = choice
    if verbose:
        print(f"[autotune] {key}: fwd ms {['%.3f' % t for t in timings_f]} bwd ms {['%.3f' % t for t in timings_b]}"
              f" -> {choice}")
    if cache_path:
        try:
            data = json.load(open(cache_path)) if os.path.exists(cache_path) else {}
        except (OSError, ValueError):
            data = {}
        data[key] = list(choice)
        with open(cache_path, "w") as f:
            json.dump(data, f, indent=1)
    return choice
