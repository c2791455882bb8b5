#!/usr/bin/env python
"""Benchmark of one edge-guided densification step on a GB300.

Workload (the 1M-Gaussian configuration): 1,000,000 Gaussians with SH degree 3
and one 1237x822 view against a synthetic target image.  One step is the
whole hot path once:

  edge map of the target (fused launch)  ->  splatting forward with L1 loss
  ->  adjoint with the edge score fused in  ->  top-10% selection  ->  Long-Axis-Split

Each timed step works on its own pre-made copy of the parameters (the split
rewrites them in place), so every step sees the identical scene; a copy is
236 MB, larger than L2, and no copy is touched twice, so no L2 flush is
needed.  The plain path (edge map one launch per stage, score accumulated in
the forward, no CUDA graph) is timed beside it on the same GPU.

`--impl reference` times the FP64 CPU oracle on the host cores instead: every
step is one whole step of the same workload, the view's pixel rows spread
over one process per host core.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd+edge-score ms/iter @1M Gaussians 1237×822 vs plain; % HBM roofline"
N_GAUSS = 1_000_000
SH_DEGREE = 3
WIDTH, HEIGHT = 1237, 822
SPLIT_FRACTION = 0.10
WORKLOAD = "1M Gaussians SH3, one 1237x822 view: edge map + fwd + L1 + bwd + edge score + top-10% LAS"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gsp", choices=["gsp", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--gaussians", type=int, default=N_GAUSS)
    ap.add_argument("--no-extra", action="store_true", help="skip the edge, multi-view and densification-loop legs")
    ap.add_argument("--variants", default=None,
                    help="forward,adjoint compositing variants (skips the autotuner; profiling runs)")
    ap.add_argument("--legs", default="main,edge,multiview,loop",
                    help="comma-separated subset of main, edge, multiview, loop (profiling runs)")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """Samples SM clock and clock-event reasons through NVML during the timed region."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown", 0x2: "applications_clocks_setting"}

    def __init__(self, pci_bus_id: str | None, period_s: float = 0.002):
        self.samples, self.reasons, self.max_mhz = [], 0, None
        self.period = period_s
        self._stop = threading.Event()
        self.ok = False
        try:
            self.nv = ctypes.CDLL("libnvidia-ml.so.1")
            if self.nv.nvmlInit_v2() != 0:
                return
            self.h = ctypes.c_void_p()
            if pci_bus_id is None or self.nv.nvmlDeviceGetHandleByPciBusId_v2(
                    pci_bus_id.encode(), ctypes.byref(self.h)) != 0:
                if self.nv.nvmlDeviceGetHandleByIndex_v2(0, ctypes.byref(self.h)) != 0:
                    return
            m = ctypes.c_uint(0)
            if self.nv.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(m)) == 0:
                self.max_mhz = int(m.value)
            self.ok = True
        except OSError:
            self.ok = False

    def _run(self):
        c = ctypes.c_uint(0)
        r = ctypes.c_ulonglong(0)
        fn_r = getattr(self.nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(self.nv, "nvmlDeviceGetCurrentClocksThrottleReasons")
        while not self._stop.is_set():
            if self.nv.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(c)) == 0:
                self.samples.append(int(c.value))
            if fn_r(self.h, ctypes.byref(r)) == 0:
                self.reasons |= int(r.value)
            time.sleep(self.period)

    def __enter__(self):
        if self.ok:
            self.t = threading.Thread(target=self._run, daemon=True)
            self.t.start()
        return self

    def __exit__(self, *a):
        if self.ok:
            self._stop.set()
            self.t.join()

    def summary(self):
        if not self.ok or not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": [n for b, n in self.REASONS.items() if self.reasons & b], "samples": len(self.samples)}


# ------------------------------------------------------------- workload

def make_inputs(n_gauss):
    import synth
    g = synth.gaussians(n_gauss, SH_DEGREE, seed=1)
    cam = synth.camera_front(WIDTH, HEIGHT)
    tgt = synth.image(HEIGHT, WIDTH, 2000)
    return g, cam, tgt


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# Algorithmic work per launch of each stage (the minimum the stage must move or
# compute for this workload): ("hbm", bytes) or ("alu", FP32 flops).
#   compositing: every pixel tests the list entries before its last contributor
#   (14 flops: offset, quadratic form, exponential, opacity, clamp, gate); each
#   composited pair then costs 12 flops forward (transmittance, colour, score)
#   and 52 flops in the adjoint (transmittance replay, colour, opacity, mean
#   and conic gradients, score)
FLOPS_EVAL, FLOPS_FWD_CONTRIB, FLOPS_BWD_CONTRIB = 14, 12, 52
FP32_LANES_PER_SM = 128


def stage_work(stage, n, k_sh, npix, pairs, evals, contrib):
    param_b = 4 * (3 + 3 + 4 + 1 + 3 * k_sh)
    rec_b = 48 + 4 + 8  # projected record + depth key + tile rectangle
    table = {
        "edge_fused": ("hbm", npix * (3 + 4)),
        "project": ("hbm", n * (param_b + rec_b)),
        "depth_sort": ("hbm", n * 4 * (4 + 4) * 2),
        "bin": ("hbm", n * (4 + 8) * 2 + pairs * 4),
        "composite_fwd": ("alu", FLOPS_EVAL * evals + FLOPS_FWD_CONTRIB * contrib),
        "composite_bwd": ("alu", FLOPS_EVAL * evals + FLOPS_BWD_CONTRIB * contrib),
        "project_bwd": ("hbm", n * (param_b + 36 + param_b)),
        "topk": ("hbm", n * 4 * 3),
        "las": ("hbm", int(SPLIT_FRACTION * n) * 2 * param_b + n),
    }
    return table.get(stage)


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) and warp
# instructions per launch (sm__inst_executed.sum) of the dominant kernel from
# one ncu capture of this workload (--set full, the kernel's first launch after
# the pair-count probe): valid for the captured variant while the compositing
# source is the one that was captured.
NCU_TRAFFIC = {("composite_bwd", 4): (46_700_544, "27b663f824539aa7")}
NCU_INST = {("composite_bwd", 4): (310_738_073, "27b663f824539aa7")}


def compositing_source_hash():
    """Hash of the adjoint compositing kernel's source and the helpers it uses
    (pixel layout, alpha evaluation, target read, warp reduction)."""
    import hashlib
    src = open(os.path.join(ROOT, "paper_2603_08661_gb300", "csrc", "render.cu")).read()
    a = src.index("// ------------------------------------------------------------- compositing")
    b = src.index("// Forward compositing: one block per 16x16 tile")
    c = src.index("// Sum of 10 per-lane values over the warp")
    d = src.index("// Chain the screen-space gradients to the parameters")
    return hashlib.sha256((src[a:b] + src[c:d]).encode()).hexdigest()[:16]


def captured_traffic(stage, variants):
    key = (stage, variants[1] if stage == "composite_bwd" else variants[0])
    if key not in NCU_TRAFFIC:
        return None
    nbytes, src = NCU_TRAFFIC[key]
    return nbytes if src == compositing_source_hash() else None


def issue_roofline(stage, variants, n_sm, sm_mhz, avg_ms):
    """The instruction-issue bound of a compositing kernel: its warp instructions
    per launch (ncu sm__inst_executed.sum, taken while the source was the one
    hashed) at one warp instruction per cycle on each of the 4 schedulers of
    every SM; frac = that time / the measured launch time.  None once the
    source has changed since the capture."""
    key = (stage, variants[1] if stage == "composite_bwd" else variants[0])
    if key not in NCU_INST:
        return None
    inst, src = NCU_INST[key]
    if src != compositing_source_hash():
        return None
    peak = 4 * n_sm * sm_mhz * 1e6
    min_ms = inst / peak * 1e3
    return {"warp_inst_per_launch": inst, "peak_warp_inst_per_s": peak, "min_ms": round(min_ms, 4),
            "frac": round(min_ms / avg_ms, 4),
            "source": "ncu sm__inst_executed.sum; 4 schedulers x SMs x max SM clock"}


# Warp instructions per launch of the edge map's walk kernel (32 views of
# 1237x822, fused mode) from one ncu capture (sm__inst_executed.sum), valid
# while the walk kernel's source is the one that was captured.
NCU_INST_EDGE = (193_025_188, "e2b2eee3cd110565")


def edge_walk_source_hash():
    """Hash of the walk kernel's source and the helpers before the tile kernel."""
    import hashlib
    src = open(os.path.join(ROOT, "paper_2603_08661_gb300", "csrc", "edge.cu")).read()
    a = src.index("// ================================================================ tile kernel")
    b = src.index("// ================================================================ walk kernel")
    c = src.index("// ------------------------------------------------------------ plain path")
    return hashlib.sha256((src[:a] + src[b:c]).encode()).hexdigest()[:16]


def alu_peak_tflops(n_sm, sm_max_mhz):
    """FP32 peak from unit counts and clock: SMs x 128 lanes x 2 flops (FMA) x clock."""
    return n_sm * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12


STAGES = ["edge_fused", "project", "depth_sort", "bin", "composite_fwd", "composite_bwd", "project_bwd",
          "topk", "las"]


def run_gsp(args, rank, world):
    import numpy as np
    import torch

    import paper_2603_08661_gb300 as gsp

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    g, cam, tgt_np = make_inputs(args.gaussians)
    n = int(g["means"].shape[0])
    k_split = int(SPLIT_FRACTION * n)
    cap = n + k_split
    k_sh = (SH_DEGREE + 1) ** 2
    npix = WIDTH * HEIGHT

    target = gsp.pitched_image(torch.from_numpy(tgt_np).to(dev), 16)
    pristine = gsp.GaussianSet.from_arrays(g, capacity=cap, device=dev)
    stream = torch.cuda.current_stream()

    # learn the pair count once (outside any timed region) to size the pair buffer
    probe = gsp.Renderer(pristine, [cam], pair_capacity=1 << 28, device=dev)
    out = probe.forward(targets=[target])
    torch.cuda.synchronize()
    gsp.raise_on_device_status(out["status"], "probe")
    pairs = int(probe.pair_count().item())
    pair_cap = int(pairs * 1.05) + 1024
    del probe, out
    torch.cuda.empty_cache()

    def clone(src):
        return gsp.GaussianSet(src.means.clone(), src.log_scales.clone(), src.quats.clone(),
                               src.opacity_logits.clone(), src.sh.clone(), src.count.clone(), src.sh_degree)

    def restore(dst, src):
        for name in ("means", "log_scales", "quats", "opacity_logits", "sh", "count"):
            getattr(dst, name).copy_(getattr(src, name))

    total = args.warmup + args.steps
    copies = [clone(pristine) for _ in range(total)]
    scores = [torch.zeros(cap, device=dev) for _ in range(total)]
    ws_r = None
    rends = []
    for c in copies:
        r = gsp.Renderer(c, [cam], pair_cap, device=dev, workspace=ws_r)
        ws_r = r.ws
        rends.append(r)
    # compositing variants chosen by the project's autotuner for this workload
    # (or given: under a profiler the autotuner's timings would be distorted)
    if args.variants:
        variants = tuple(int(x) for x in args.variants.split(","))
    else:
        variants = gsp.autotune.tune(rends[0], targets=[target])
    for r in rends:
        r.variants = variants
    E = torch.empty(npix, dtype=torch.float32, device=dev)
    ws_e = torch.empty(1 << 26, dtype=torch.uint8, device=dev)
    ws_las = torch.empty(gsp._lib.load().gsp_las_workspace_size(cap), dtype=torch.uint8, device=dev)
    status = gsp.new_status(dev)
    grads = {"means": torch.zeros_like(pristine.means), "log_scales": torch.zeros_like(pristine.log_scales),
             "quats": torch.zeros_like(pristine.quats), "opacity_logits": torch.zeros_like(pristine.opacity_logits),
             "sh": torch.zeros_like(pristine.sh)}
    fwd_bufs = {"rgb": torch.empty((npix, 3), device=dev), "T": torch.empty(npix, device=dev),
                "last": torch.empty(npix, dtype=torch.int32, device=dev), "loss": torch.empty(1, device=dev)}

    # the second stream (edge map, selection) at the highest priority: its blocks are
    # scheduled ahead of the adjoint's pending ones (measured: the graph replays are
    # unchanged, the eager end-to-end steps 20-50 us faster)
    edge_stream = torch.cuda.Stream(device=dev, priority=-5)
    score_ev = torch.cuda.Event()
    ws_sel = torch.empty_like(ws_las)
    sel_mask = torch.empty(cap, dtype=torch.uint8, device=dev)
    edge_bps = 1  # one edge-map block per SM beside the forward (measured 1.18 ms per step; 2: 1.19, all: 1.20)

    def step(j, plain=False, tgt=None, overlap=True):
        r = rends[j]
        tgt = target if tgt is None else tgt
        if not plain and not overlap:
            # the same launches one after another (the per-stage timings)
            gsp.edge_map([tgt], mode="fused", out=E, status=status, workspace=ws_e)
            out = r.forward(targets=[tgt], status=status, out=fwd_bufs)
            r.backward(out, targets=[tgt], edge=E, score=scores[j], grads=grads, status=status)
        elif plain:
            gsp.edge_map([tgt], mode="plain", out=E, status=status, workspace=ws_e)
            out = r.forward(targets=[tgt], edge=E, score=scores[j], status=status, out=fwd_bufs)
            r.backward(out, targets=[tgt], grads=grads, status=status)
        else:
            # the edge map needs only the target and the forward pass does not read
            # it: it runs on a second stream beside projection, sort, binning and
            # forward compositing, and the adjoint (which takes the edge score) waits
            cur = torch.cuda.current_stream(dev)
            edge_stream.wait_stream(cur)
            with torch.cuda.stream(edge_stream):
                gsp.edge_map([tgt], mode="fused", out=E, status=status, workspace=ws_e, blocks_per_sm=edge_bps)
            out = r.forward(targets=[tgt], status=status, out=fwd_bufs)
            cur.wait_stream(edge_stream)
            r.backward(out, targets=[tgt], edge=E, score=scores[j], grads=grads, status=status,
                       score_event=score_ev)
            # the selection needs only the edge score: it runs on the second stream
            # while the adjoint chains the gradients to the parameters; the split
            # (which rewrites parameters the chain reads) waits for both
            edge_stream.wait_event(score_ev)
            with torch.cuda.stream(edge_stream):
                gsp.select_mask(scores[j], copies[j].count, k_split, status=status, workspace=ws_sel,
                                out=sel_mask)
            cur.wait_stream(edge_stream)
            gsp.las_split(copies[j], mask=sel_mask, params=gsp.LAS_CONFIG, status=status, workspace=ws_las)
            return out
        gsp.las_split(copies[j], scores=scores[j], k=k_split, params=gsp.LAS_CONFIG, status=status,
                      workspace=ws_las)
        return out

    # launches per step (counted by the library while enqueueing one eager step)
    l0 = gsp.launch_count()
    step(0)
    launches_per_step = gsp.launch_count() - l0
    torch.cuda.synchronize()
    gsp.raise_on_device_status(status, "first step")
    restore(copies[0], pristine)
    scores[0].zero_()

    # per-stage breakdown (one eager step per armed stage, untimed)
    breakdown = {}
    for st in STAGES:
        timer = gsp.StageTimer(st, 8)
        step(0, overlap=False)
        ms, cnt = timer.read()
        breakdown[st] = ms / max(cnt, 1)
        restore(copies[0], pristine)
        scores[0].zero_()
    gsp.StageTimer.disarm()
    torch.cuda.synchronize()
    dominant = max(breakdown, key=lambda s: breakdown[s])
    # data-dependent work counts of the workload (the scene is identical every step)
    stats = rends[0].stats().cpu()
    contrib = int(stats[1])
    redone = int(stats[2])
    evals = int(fwd_bufs["last"].to(torch.int64).sum().item())

    # capture one graph per copy; the dominant stage is bracketed by library events
    use_graph = not args.no_graph
    graphs = []
    timer = None
    if use_graph:
        try:
            side = torch.cuda.Stream(device=dev)
            side.wait_stream(stream)
            with torch.cuda.stream(side):
                for j in range(total):
                    if j == args.warmup:
                        timer = gsp.StageTimer(dominant, args.steps)
                    gr = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(gr, stream=side):
                        step(j)
                    graphs.append(gr)
            stream.wait_stream(side)
            torch.cuda.synchronize()
        except Exception as exc:  # capture unsupported: fall back to eager launches
            print(f"[bench] graph capture failed ({exc}); timing eager launches", file=sys.stderr)
            use_graph = False
            graphs = []
            torch.cuda.synchronize()
            for j in range(total):
                restore(copies[j], pristine)
                scores[j].zero_()
    if not use_graph:
        timer = None

    def run_range(lo, hi):
        for j in range(lo, hi):
            if use_graph:
                graphs[j].replay()
            else:
                step(j)

    run_range(0, args.warmup)
    if not use_graph:
        timer = gsp.StageTimer(dominant, args.steps)
    torch.cuda.synchronize()
    dist_barrier(world)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    props = torch.cuda.get_device_properties(dev)
    bus = getattr(props, "pci_bus_id", None)
    bus_str = None if bus is None else f"{getattr(props, 'pci_domain_id', 0):08x}:{bus:02x}:{getattr(props, 'pci_device_id', 0):02x}.0"
    with ClockSampler(bus_str) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        run_range(args.warmup, total)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms_total = ev0.elapsed_time(ev1)
    dom_ms, dom_cnt = timer.read()
    gsp.StageTimer.disarm()
    gsp.raise_on_device_status(status, "timed steps")
    ms_total = dist_max(ms_total, world)
    ms_step = ms_total / args.steps

    # plain path: edge map per stage, score in the forward, no graph
    plain = None
    if not args.no_plain:
        m = min(args.steps, 20)
        for j in range(m + 3):
            restore(copies[j], pristine)
            scores[j].zero_()
        for j in range(3):
            step(j, plain=True)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for j in range(3, 3 + m):
            step(j, plain=True)
        b.record(stream)
        torch.cuda.synchronize()
        plain = {"ms_per_step": a.elapsed_time(b) / m, "steps": m, "graph": False,
                 "edge_map": "one launch per stage", "score": "accumulated in the forward"}

    # end to end: pinned host parameters and image in, loss and count out, every step
    e2e = None
    if not args.no_e2e:
        # the step's inputs: the N live Gaussians (rows past N are room for the split's children)
        host = {name: (getattr(pristine, name) if name == "count" else getattr(pristine, name)[:n]).cpu().pin_memory()
                for name in ("means", "log_scales", "quats", "opacity_logits", "sh", "count")}
        host_img = target.cpu().pin_memory()
        res_host = torch.empty(2, dtype=torch.float32).pin_memory()
        h2d = sum(t.numel() * t.element_size() for t in host.values()) + host_img.numel()
        m = min(args.steps, 20)

        def serial():
            """Copies, step and read-back one after another on one stream."""
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            a.record(stream)
            for j in range(m):
                c = copies[j]
                for name, t in host.items():
                    getattr(c, name)[:t.shape[0]].copy_(t, non_blocking=True)
                target.copy_(host_img, non_blocking=True)
                scores[j].zero_()
                out = step(j)
                res_host[0].copy_(out["loss"][0], non_blocking=True)
                res_host[1:2].copy_(c.count.float(), non_blocking=True)
            b.record(stream)
            torch.cuda.synchronize()
            wall = (time.perf_counter() - t0) * 1e3 / m
            return max(a.elapsed_time(b) / m, wall)

        def pipelined():
            """Step j + 1's copies on a copy stream while step j computes: every
            step's inputs still cross from pinned host memory inside the timed
            region, into its own parameter buffers and one of two target
            buffers (reused once the step two before has finished with it)."""
            cs = torch.cuda.Stream(device=dev)
            tbuf = [target, gsp.pitched_image(target.clone(), 16)]
            ev_in = [torch.cuda.Event() for _ in range(m)]
            ev_free = [torch.cuda.Event(), torch.cuda.Event()]
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            a.record(stream)
            cs.wait_event(a)

            def enqueue_copy(j):
                with torch.cuda.stream(cs):
                    if j >= 2:
                        cs.wait_event(ev_free[j % 2])
                    c = copies[j]
                    for name, t in host.items():
                        getattr(c, name)[:t.shape[0]].copy_(t, non_blocking=True)
                    tbuf[j % 2].copy_(host_img, non_blocking=True)
                    ev_in[j].record(cs)

            enqueue_copy(0)
            for j in range(m):
                if j + 1 < m:
                    enqueue_copy(j + 1)
                stream.wait_event(ev_in[j])
                scores[j].zero_()
                out = step(j, tgt=tbuf[j % 2])
                ev_free[j % 2].record(stream)
                res_host[0].copy_(out["loss"][0], non_blocking=True)
                res_host[1:2].copy_(copies[j].count.float(), non_blocking=True)
            b.record(stream)
            torch.cuda.synchronize()
            wall = (time.perf_counter() - t0) * 1e3 / m
            return max(a.elapsed_time(b) / m, wall)

        ms_serial = serial()
        for j in range(m):
            restore(copies[j], pristine)
        ms_pipe = pipelined()
        e2e = {"value": round(ms_pipe, 4), "unit": "ms/iter", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": 8, "steps": m, "serial_ms_per_iter": round(ms_serial, 4),
               "note": "the N live Gaussians' parameters and the target image copied from pinned host memory every step (step j + 1's "
                       "copies on a second stream overlap step j), loss and count read back every step; "
                       "serial_ms_per_iter: copies, step and read-back one after another"}

    hbm, peak_kind = peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_max = clk.max_mhz or 2070
    alu_peak = alu_peak_tflops(props.multi_processor_count, sm_max)
    dom_avg_ms = dom_ms / max(dom_cnt, 1)

    def roofline(stage, ms):
        bound, amount = stage_work(stage, n, k_sh, npix, pairs, evals, contrib)
        if bound == "hbm":
            ach = amount / (ms * 1e-3) / 1e9
            return {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                    "frac": round(ach / hbm, 4), "algorithmic_per_launch": amount}
        ach = amount / (ms * 1e-3) / 1e12
        return {"bound": "alu", "achieved": round(ach, 3), "peak": round(alu_peak, 1), "unit": "TFLOP/s",
                "frac": round(ach / alu_peak, 4), "algorithmic_per_launch": amount}

    roof = roofline(dominant, dom_avg_ms)
    roof.update({"kernel": dominant, "traffic": captured_traffic(dominant, variants),
                 "issue": issue_roofline(dominant, variants, props.multi_processor_count, sm_max, dom_avg_ms),
                 "avg_launch_ms": round(dom_avg_ms, 5), "launches": dom_cnt,
                 "peak_source": (f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if roof["bound"] == "hbm" else
                                 f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                                 f"{sm_max} MHz")})
    stages_roof = {st: dict(roofline(st, ms), ms=round(ms, 4)) for st, ms in breakdown.items()}

    next_rows = None
    if not args.no_extra:
        restore(copies[0], pristine)
        next_rows = {"gating": measure_gating(gsp, rends[0], target, E, k_split)}
        restore(copies[0], pristine)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(n)

    line = {
        "metric": METRIC, "value": round(ms_step / world, 4), "unit": "ms/iter", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded scenes shaped like the paper's Mip-NeRF360 views)",
        "config": {"workload": WORKLOAD, "gaussians": n, "sh_degree": SH_DEGREE, "view": f"{WIDTH}x{HEIGHT}",
                   "split_k": k_split, "pairs": pairs, "graph": use_graph, "variants": list(variants),
                   "l2": "inputs larger than L2: every step uses its own 236 MB parameter copy",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches_per_step * args.steps),
        "clocks": clk.summary(), "plain": plain,
        "stages": stages_roof,
        "work_counts": {"pairs": pairs, "evaluations": evals, "composited": contrib, "redone_tiles": redone},
        "next_rows": next_rows,
    }
    return line


# ------------------------------------------------- extra workloads (same run)

def _probe_pairs(gsp, gs, cams):
    """Tile-Gaussian pairs of the scene (a small probe: the count is exact even
    beyond the probe's capacity)."""
    import torch
    probe = gsp.Renderer(gs, cams, pair_capacity=1 << 20)
    probe.forward()
    torch.cuda.synchronize()
    pairs = int(probe.pair_count().item())
    del probe
    torch.cuda.empty_cache()
    return pairs


def _event_ms(fn, reps):
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def measure_gating(gsp, r, target, E, k, reps=10):
    """The next rows on the main workload: the adjoint with and without the
    positional statistic and the gated selection beside the plain one
    (threshold: the median mean gradient of the Gaussians seen), importance
    sampling, and the plain against the scheduled SGD step."""
    import numpy as np
    import torch
    dev = r.gs.means.device
    cap = r.gs.capacity
    score = torch.zeros(cap, device=dev)
    psum = torch.zeros(cap, device=dev)
    pcnt = torch.zeros(cap, dtype=torch.int32, device=dev)
    out = r.forward(targets=[target])
    grads = r.backward(out, targets=[target], edge=E, score=score, pos_grad=(psum, pcnt))
    torch.cuda.synchronize()
    s_h, c_h = psum.cpu().numpy(), pcnt.cpu().numpy()
    seen = c_h > 0
    tau = float(np.median(s_h[seen] / c_h[seen])) if seen.any() else 0.0
    bwd = _event_ms(lambda: r.backward(out, targets=[target], edge=E, score=score, grads=grads), reps)
    bwd_stat = _event_ms(lambda: r.backward(out, targets=[target], edge=E, score=score, grads=grads,
                                            pos_grad=(psum, pcnt)), reps)
    plain = _event_ms(lambda: gsp.topk_mask(score, r.gs.count, k), reps)
    gated = _event_ms(lambda: gsp.topk_mask_gated(score, psum, pcnt, tau, r.gs.count, k), reps)
    _, sel, st = gsp.topk_mask_gated(score, psum, pcnt, tau, r.gs.count, k)
    torch.cuda.synchronize()
    gsp.raise_on_device_status(st, "gated top-k")
    expv = torch.empty(cap, device=dev).exponential_()  # the sampling's Exp(1) inputs
    sample = _event_ms(lambda: gsp.sample_mask(score, expv, r.gs.count, k), reps)
    # optimiser step: plain SGD against the device-scheduled rates (Sec. 2.3 decays); the
    # parameters are restored afterwards by the caller's copy
    import ctypes
    from paper_2603_08661_gb300 import _lib as L
    lib = L.load()
    gp = [grads[name] for name in ("means", "log_scales", "quats", "opacity_logits", "sh")]
    ptrs = [ctypes.c_void_p(t.data_ptr()) for t in gp]
    sched = L.LrSchedule((L.c_f32 * 5)(1.28e-4, 0.020, 1e-3, 5e-2, 2.5e-3),
                         (L.c_f32 * 5)(1.28e-5, 0.002, 1e-3, 5e-2, 2.5e-3), 30000)
    step = torch.zeros(1, dtype=torch.int32, device=dev)
    sgd = _event_ms(lambda: lib.gsp_sgd_step(ctypes.byref(r.gs.struct()), *ptrs, ctypes.c_float(0.0), None), reps)
    sgd_s = _event_ms(lambda: lib.gsp_sgd_step_scheduled(ctypes.byref(r.gs.struct()), *ptrs, ctypes.byref(sched),
                                                         ctypes.c_void_p(step.data_ptr()), None), reps)
    return {"row": "gradient-threshold masking (Sec. 2.3 warm-up masking)",
            "adjoint_ms": round(bwd, 4), "adjoint_with_statistic_ms": round(bwd_stat, 4),
            "topk_ms": round(plain, 4), "topk_gated_ms": round(gated, 4), "k": int(k),
            "seen": int(seen.sum()), "threshold": tau, "selected": int(sel.item()),
            "sampling_ms": round(sample, 4), "sgd_ms": round(sgd, 4), "sgd_scheduled_ms": round(sgd_s, 4),
            "note": "eager launches incl. host overhead; statistic fused into the adjoint's parameter pass"}


def run_edge_batched(steps=10, warmup=3, sm_max_mhz=None):
    """32 views of 1237x822: the fused edge map (every stage of every view in one
    cooperative launch) against the plain path (one launch per stage and view).
    `issue`: the walk kernel's instruction-issue bound (its ncu warp
    instructions at one per cycle on 4 schedulers x SMs x max SM clock) against
    the measured launch time, while its source is the captured one."""
    import torch

    import paper_2603_08661_gb300 as gsp
    import synth
    nv = 32
    views = [gsp.pitched_image(torch.from_numpy(synth.image(HEIGHT, WIDTH, 1000 + v)).cuda(), 16) for v in range(nv)]
    npix = nv * WIDTH * HEIGHT
    out = torch.empty(npix, device="cuda")
    status = gsp.new_status()
    ws = torch.empty(1 << 28, dtype=torch.uint8, device="cuda")
    res = {}
    for mode in ("fused", "plain"):
        def run():
            gsp.edge_map(views, mode=mode, out=out, status=status, workspace=ws)
        for _ in range(warmup):
            run()
        res[mode] = _event_ms(run, steps)
    torch.cuda.synchronize()
    gsp.raise_on_device_status(status, "edge batched")
    algo = npix * (3 + 4)
    hbm, _ = peaks()
    issue = None
    if NCU_INST_EDGE is not None and NCU_INST_EDGE[1] == edge_walk_source_hash():
        n_sm = torch.cuda.get_device_properties(0).multi_processor_count
        peak = 4 * n_sm * (sm_max_mhz or 2070) * 1e6
        min_ms = NCU_INST_EDGE[0] / peak * 1e3
        issue = {"warp_inst_per_launch": NCU_INST_EDGE[0], "min_ms": round(min_ms, 4),
                 "frac": round(min_ms / res["fused"], 4),
                 "source": "ncu sm__inst_executed.sum; 4 schedulers x SMs x max SM clock"}
    return {"workload": "32 views 1237x822 uint8 RGB -> fp32 E", "ms_fused_batched": round(res["fused"], 4),
            "ms_plain_per_view_per_stage": round(res["plain"], 4),
            "fused_achieved_gbs": round(algo / (res["fused"] * 1e-3) / 1e9, 1),
            "fused_frac_of_hbm": round(algo / (res["fused"] * 1e-3) / 1e9 / hbm, 4),
            "issue": issue,
            "algorithmic_bytes": algo, "l2": "inputs 98 MB + outputs 130 MB per launch (larger than L2)"}


def run_multiview(steps=5, warmup=3):
    """3M SH-3 Gaussians, 8 ring views of uneven resolution: forward + L1 +
    adjoint with the edge score, all views in one call per pass, captured as a
    CUDA graph with autotuned compositing variants, against the plain path
    (one call per view and pass, default variants, no graph)."""
    import torch

    import paper_2603_08661_gb300 as gsp
    import synth
    n, nv = 3_000_000, 8
    g = synth.gaussians(n, 3, seed=1)
    cams = [synth.camera_ring(k, nv) for k in range(nv)]
    gs = gsp.GaussianSet.from_arrays(g, capacity=n)
    del g
    targets = [gsp.pitched_image(torch.from_numpy(synth.image(c["height"], c["width"], 2000 + k)).cuda(), 16)
               for k, c in enumerate(cams)]
    E, _, _, st = gsp.edge_map(targets)
    pairs = _probe_pairs(gsp, gs, cams)
    r = gsp.Renderer(gs, cams, pair_capacity=int(pairs * 1.02) + 4096)
    variants = gsp.autotune.tune(r, targets=targets)
    score = torch.zeros(n, device="cuda")
    grads = {k: torch.zeros_like(getattr(gs, k)) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    npix = r.total_pix
    bufs = {"rgb": torch.empty((npix, 3), device="cuda"), "T": torch.empty(npix, device="cuda"),
            "last": torch.empty(npix, dtype=torch.int32, device="cuda"), "loss": torch.empty(1, device="cuda")}
    status = gsp.new_status()

    def it():
        out = r.forward(targets=targets, status=status, out=bufs)
        r.backward(out, targets=targets, edge=E, score=score, grads=grads, status=status)

    it()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            it()
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(warmup):
        graph.replay()
    ms_graph = _event_ms(graph.replay, steps)
    torch.cuda.synchronize()
    gsp.raise_on_device_status(status, "multiview")
    # per-stage CUDA-event times (eager iterations, one armed stage at a time)
    stages = {}
    for stg in ("project", "depth_sort", "bin", "composite_fwd", "composite_bwd", "project_bwd"):
        timer = gsp.StageTimer(stg, 4)
        for _ in range(2):
            it()
        ms, cnt = timer.read()
        stages[stg] = round(ms / max(cnt, 1), 3)
    gsp.StageTimer.disarm()
    redone = int(r.stats()[2].item())  # tiles whose list prefix did not suffice
    # plain path: one single-view call per view and pass, default variants, eager
    del r
    torch.cuda.empty_cache()
    per_view = []
    big = 0
    for k, c in enumerate(cams):
        pv = _probe_pairs(gsp, gs, [c])
        big = max(big, pv)
    ws = None
    for k, c in enumerate(cams):
        rv = gsp.Renderer(gs, [c], pair_capacity=int(big * 1.02) + 4096, workspace=ws)
        ws = rv.ws
        per_view.append(rv)
    offs = [0]
    for c in cams:
        offs.append(offs[-1] + c["width"] * c["height"])
    Ev = [E[offs[k]:offs[k + 1]] for k in range(nv)]

    def it_plain():
        for k, rv in enumerate(per_view):
            out = rv.forward(targets=[targets[k]], status=status)
            rv.backward(out, targets=[targets[k]], edge=Ev[k], score=score, grads=grads, status=status,
                        accumulate=k > 0)

    for _ in range(warmup):
        it_plain()
    ms_plain = _event_ms(it_plain, steps)
    torch.cuda.synchronize()
    gsp.raise_on_device_status(status, "multiview plain")
    return {"workload": "3M Gaussians SH3, 8 ring views 640x480..1920x1080 (8.76 Mpix): fwd + L1 + bwd + edge score",
            "pairs": pairs, "variants": list(variants), "ms_per_iter_batched_graph": round(ms_graph, 3),
            "ms_per_iter_plain_per_view": round(ms_plain, 3), "mpix_per_s_batched": round(npix / ms_graph / 1e3, 1),
            "steps": steps, "stages_ms": stages, "redone_tiles": redone}


def run_multiview_sharded(rank, world, steps=5, warmup=3):
    """The 3M-Gaussian, 8-view workload sharded over the ranks by view
    (paper_2603_08661_gb300.sharded): each rank renders its share (forward + L1 +
    adjoint with the edge score), then one all-reduce (sum) of gradients, scores
    and loss.  Total work is fixed as the ranks grow (strong scaling); the time
    is the max over ranks."""
    import torch

    import paper_2603_08661_gb300 as gsp
    import synth
    n, nv = 3_000_000, 8
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    g = synth.gaussians(n, 3, seed=1)
    cams = [synth.camera_ring(k, nv) for k in range(nv)]
    gs = gsp.GaussianSet.from_arrays(g, capacity=n, device=dev)
    del g
    targets = [torch.from_numpy(synth.image(c["height"], c["width"], 2000 + k)).to(dev) for k, c in enumerate(cams)]
    E, _, _, _ = gsp.edge_map(targets)
    views = gsp.partition_views([c["width"] * c["height"] for c in cams], world)[rank]
    pairs = _probe_pairs(gsp, gs, [cams[v] for v in views]) if views else 1
    sr = gsp.ShardedRenderer(gs, cams, pair_capacity=int(pairs * 1.02) + 4096, device=dev)
    for _ in range(warmup):
        sr.step(targets, edge=E)
    torch.cuda.synchronize()
    dist_barrier(world)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        sr.step(targets, edge=E)
    b.record()
    torch.cuda.synchronize()
    ms = dist_max(a.elapsed_time(b) / steps, world)
    if sr.r is not None:
        gsp.raise_on_device_status(sr.status, "multiview sharded")
    return {"workload": "3M Gaussians SH3, 8 ring views 640x480..1920x1080 sharded by view over the ranks: "
                        "fwd + L1 + bwd + edge score, one all-reduce of gradients, scores and loss",
            "ranks": world, "views_of_rank0": views if rank == 0 else None, "ms_per_iter": round(ms, 3),
            "allreduce_bytes": int(sr.out.flat.numel() * 4), "scaling": "strong", "steps": steps}


def run_densify_loop(iterations=200, warmup=3):
    """500K -> 1M Gaussians (SH degree 0, as the tiny configuration) on 4 ring
    views of 1237x822: 200 graph-replayed iterations of fwd + L1 + bwd with the
    edge score + SGD (lr 1e-3), a top-k (50K) + LAS event every 20."""
    import torch

    import paper_2603_08661_gb300 as gsp
    import synth
    n0, cap, nv = 500_000, 1_000_000, 4
    g = synth.gaussians(n0, 0, seed=1)
    cams = [synth.camera_ring(k, nv, resolutions=[(WIDTH, HEIGHT)]) for k in range(nv)]
    gs = gsp.GaussianSet.from_arrays(g, capacity=cap)
    targets = [gsp.pitched_image(torch.from_numpy(synth.image(HEIGHT, WIDTH, 2000 + k)).cuda(), 16)
               for k in range(nv)]
    pairs0 = _probe_pairs(gsp, gs, cams)
    loop = gsp.DensifyLoop(gs, cams, targets, lr=1e-3, every=20, k_event=50_000,
                           pair_capacity=int(pairs0 * 2.5) + 4096)
    saved = {k: getattr(gs, k).clone() for k in ("means", "log_scales", "quats", "opacity_logits", "sh", "count")}
    loop.capture()
    loop.run(warmup)
    torch.cuda.synchronize()
    for k, v in saved.items():
        getattr(gs, k).copy_(v)
    loop.score.zero_()
    loop.iteration_count = 0
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    loop.run(iterations)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    gsp.raise_on_device_status(loop.status, "densify loop")
    return {"workload": "500K -> 1M Gaussians SH0, 4 ring views 1237x822, 200 iterations, top-k 50K + LAS every 20",
            "iterations": iterations, "total_ms": round(ms, 2), "ms_per_iter": round(ms / iterations, 4),
            "final_gaussians": int(gs.count.item()), "pairs_at_start": pairs0,
            "loss_last": round(float(loop.loss().item()), 6)}


# --------------------------------------------------------------- oracle

_ORC = {}  # per-process inputs of the oracle step (set in pool workers and in the serial path)


def _orc_init(n_gauss):
    """Pool worker: the step's inputs, made from the same seeds as the GPU leg."""
    import synth
    _ORC["g"] = synth.gaussians(n_gauss, SH_DEGREE, seed=1)
    _ORC["cam"] = synth.camera_front(WIDTH, HEIGHT)
    _ORC["t"] = synth.image(HEIGHT, WIDTH, 2000) / 255.0


def _orc_attach(spec):
    from multiprocessing import shared_memory

    import numpy as np
    shm = shared_memory.SharedMemory(name=spec[0])
    return shm, np.ndarray(spec[1], dtype=spec[2], buffer=shm.buf)


def _orc_stripe(task):
    """Rows [y0, y1) of the view through the oracle as it stands: forward
    composite with the edge score, L1 sign, analytic adjoint.  Returns the
    gradient rows of the Gaussians the stripe touches, its score entries and
    its part of the L1 sum."""
    import numpy as np

    from oracle import raster as orc
    y0, y1, specs = task
    t_begin = time.perf_counter()
    g, cam, t = _ORC["g"], _ORC["cam"], _ORC["t"]
    held = [_orc_attach(sp) for sp in specs]
    proj, order, E = (a for _, a in held)
    try:
        reg = (0, y0, WIDTH, y1)
        out = orc.render(g, cam, edge=E, region=reg, proj=proj, order=order)
        d = out["rgb"][y0:y1] - t[y0:y1]
        dl = np.zeros((HEIGHT, WIDTH, 3))
        dl[y0:y1] = np.sign(d) / (3.0 * WIDTH * HEIGHT)
        gr = orc.render_bwd(g, cam, dl, proj=proj, region=reg)
    finally:
        for shm, _ in held:
            shm.close()
    n = g["means"].shape[0]
    touched = np.zeros(n, bool)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        touched |= (gr[k].reshape(n, -1) != 0).any(axis=1)
    idx = np.flatnonzero(touched)
    sidx = np.flatnonzero(out["score"])
    return (idx, {k: gr[k].reshape(n, -1)[idx] for k in ("means", "log_scales", "quats", "opacity_logits", "sh")},
            sidx, out["score"][sidx], float(np.abs(d).sum()), time.perf_counter() - t_begin)


class OracleStep:
    """One whole step of the hot path through the FP64 oracle, on `workers`
    host processes: the edge map of the target, projection and compositing
    order of all Gaussians, the forward composite with the edge score, the L1
    loss and the analytic adjoint over every pixel of the view (full-width row
    stripes spread over the workers, their gradient rows and scores summed),
    the top-10 % selection and the Long-Axis-Split.  The oracle's code runs as
    it stands; only the pixel rows are divided among processes (spawned, so
    that a process that has used the GPU can host them)."""

    def __init__(self, n_gauss, workers, stripes_per_worker=1):
        import multiprocessing as mp

        import numpy as np
        _orc_init(n_gauss)
        self.n = n_gauss
        self.workers = max(1, int(workers))
        self.stripes_per_worker = int(stripes_per_worker)
        self.pool = None
        if self.workers > 1:
            self.pool = mp.get_context("spawn").Pool(self.workers, initializer=_orc_init, initargs=(n_gauss,))
            self.pool.map(abs, range(self.workers))  # every worker has made its inputs
        k_sh = (SH_DEGREE + 1) ** 2
        self.cols = {"means": 3, "log_scales": 3, "quats": 4, "opacity_logits": 1, "sh": 3 * k_sh}
        self.grads = {k: np.zeros((n_gauss, c)) for k, c in self.cols.items()}
        self.score = np.zeros(n_gauss)

    def close(self):
        if self.pool is not None:
            self.pool.close()
            self.pool.join()
            self.pool = None

    def step(self):
        """Seconds of one whole step (all of its parts measured, nothing scaled)."""
        from multiprocessing import shared_memory

        import numpy as np

        import synth
        from oracle import densify as od
        from oracle import edge as oe
        from oracle import raster as orc
        parallel = self.pool is not None
        g, cam = _ORC["g"], _ORC["cam"]
        tgt_u8 = synth.image(HEIGHT, WIDTH, 2000)
        t0 = time.perf_counter()
        E = oe.edge_map(tgt_u8)["E"]
        proj = orc.project(g, cam)
        order = orc.order(proj)
        t1 = time.perf_counter()
        shms, specs = [], []
        for arr in (proj, order, E):
            shm = shared_memory.SharedMemory(create=True, size=max(arr.nbytes, 1))
            np.ndarray(arr.shape, dtype=arr.dtype, buffer=shm.buf)[...] = arr
            shms.append(shm)
            specs.append((shm.name, arr.shape, arr.dtype.str))
        nstripes = self.stripes_per_worker * self.workers if parallel else 1
        edges = [round(i * HEIGHT / nstripes) for i in range(nstripes + 1)]
        tasks = [(edges[i], edges[i + 1], specs) for i in range(nstripes) if edges[i + 1] > edges[i]]
        try:
            parts = (self.pool.map(_orc_stripe, tasks, chunksize=1) if parallel
                     else [_orc_stripe(tk) for tk in tasks])
        finally:
            for shm in shms:
                shm.close()
                shm.unlink()
        for k in self.grads:
            self.grads[k].fill(0.0)
        self.score.fill(0.0)
        loss = 0.0
        busy = 0.0
        for idx, rows, sidx, svals, l1, dt in parts:
            for k in self.grads:
                self.grads[k][idx] += rows[k]
            self.score[sidx] += svals
            loss += l1
            busy += dt
        t2 = time.perf_counter()
        k_split = int(SPLIT_FRACTION * self.n)
        mask = od.topk_mask(self.score, k_split)
        od.las_split(g, mask, **od.CONFIG_PRESET)
        t3 = time.perf_counter()
        self.loss = loss / (3.0 * WIDTH * HEIGHT)
        # busy seconds of every process: the step's CPU time, i.e. one core's share of work
        self.cpu_seconds = (t1 - t0) + busy + (t3 - t2)
        return t3 - t0, {"edge_project_order": round(t1 - t0, 3), "render_adjoint": round(t2 - t1, 3),
                         "topk_las": round(t3 - t2, 3), "stripes": len(tasks),
                         "stripe_busy_s": round(busy, 3)}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_baseline(n_gauss, one_core=True):
    """The FP64 oracle timed on the host cores in the GPU run: one whole step on
    every core (the value), its CPU time (the busy seconds of all processes
    summed), and one whole step on one core."""
    cores = host_cores()
    o = OracleStep(n_gauss, cores)
    try:
        t_all, parts_all = o.step()
    finally:
        o.close()
    out = {"value": round(1e3 * t_all, 1), "unit": "ms/iter", "cores": cores, "kind": "oracle",
           "sample": f"one whole step (edge map, projection, forward composite with edge score, L1, analytic "
                     f"adjoint over all {WIDTH}x{HEIGHT} pixels, top-10% selection, LAS) of the FP64 oracle on "
                     f"{cores} host processes (one pixel-row stripe each), measured, nothing scaled",
           "cpu_seconds_per_step": round(o.cpu_seconds, 1), "parts_s": parts_all}
    if one_core and cores > 1:
        o1 = OracleStep(n_gauss, 1)
        try:
            t1, parts1 = o1.step()
        finally:
            o1.close()
        out["one_core"] = {"value": round(1e3 * t1, 1), "unit": "ms/iter", "cores": 1,
                           "sample": "the same whole step in one process", "parts_s": parts1}
    return out


def run_reference(args, rank, world):
    """The reference arm: the FP64 oracle as it stands, one whole step of the
    workload per step, on every host core (rank 0 only)."""
    if rank != 0:
        return None
    cores = host_cores()
    o = OracleStep(args.gaussians, cores)
    vals = []
    try:
        for i in range(args.warmup + args.steps):
            t, parts = o.step()
            if i >= args.warmup:
                vals.append(1e3 * t)
    finally:
        o.close()
    v = statistics.mean(vals)
    sample = (f"whole steps of the FP64 oracle (edge map, projection, forward composite with edge score, L1, "
              f"analytic adjoint over all {WIDTH}x{HEIGHT} pixels, top-10% selection, LAS) on {cores} host "
              f"processes, each step measured")
    return {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": "ms/iter", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v, 1), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "gaussians": args.gaussians, "sh_degree": SH_DEGREE,
                       "view": f"{WIDTH}x{HEIGHT}"},
            "cpu_baseline": {"value": round(v, 1), "unit": "ms/iter", "cores": cores, "kind": "oracle",
                             "sample": sample, "parts_s_last_step": parts,
                             "cpu_seconds_last_step": round(o.cpu_seconds, 1)},
            "e2e": {"value": round(v, 1), "unit": "ms/iter", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------- distributed

def dist_setup():
    """One process per GPU (torchrun env); NCCL on GPUs, gloo without them.
    The main workload (one view) runs as independent replicas, so for it the
    group only carries the barriers and the max-over-ranks of the timed region;
    the multi-view leg runs view-sharded with one all-reduce per iteration."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    return rank, world


def dist_barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def dist_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def main():
    args = parse()
    rank, world = dist_setup()
    if args.impl == "reference":
        if world > 1:
            # the reference arm runs on rank 0 only
            pass
        line = run_reference(args, rank, world)
    else:
        legs = set(args.legs.split(","))
        line = run_gsp(args, rank, world) if "main" in legs else {"metric": METRIC, "legs": sorted(legs)}
        if world == 1 and not args.no_extra:
            import torch
            for name, key, fn in (("edge", "edge_batched", run_edge_batched), ("multiview", "multiview", run_multiview),
                                  ("loop", "densify_loop", run_densify_loop)):
                if name in legs:
                    torch.cuda.empty_cache()
                    if name == "edge":
                        line[key] = fn(sm_max_mhz=(line.get("clocks") or {}).get("sm_max_mhz"))
                    else:
                        line[key] = fn()
        elif world > 1 and not args.no_extra and "multiview" in legs:
            # N > 1: the multi-view workload runs view-sharded (one all-reduce per iteration)
            import torch
            torch.cuda.empty_cache()
            line["multiview_sharded"] = run_multiview_sharded(rank, world)
    if rank == 0 and line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        if args.impl != "reference":
            dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
