"""Device-resident densification loop around the edge-guided densification.

One iteration: splatting forward over the fixed views with the L1 loss, the
adjoint with the edge score (Sec. 1, "Edge-Score importance") accumulated in
the same pass, and a plain SGD step on every parameter.  Every `every`
iterations a densification event takes the top-k Gaussians by accumulated
edge score (or samples k with probabilities proportional to it, selection =
"sample"), splits them with the Long-Axis-Split (Sec. 2.2, Alg. 1-2; the
paper's preset by default) into
the free capacity rows, and clears the scores.  The edge maps of the fixed
target views (Sec. 2.1) are computed once, in one fused launch.

With grad_threshold set, the adjoint also accumulates the positional
statistic of the gradient-threshold masking, and every event after the first
`warmup_events` (three: Sec. 2.3, "Global Warm-up Phase") selects only among
the Gaussians whose mean positional gradient reaches the threshold; the
statistic is cleared with the scores after each event.  The graph driver
captures the threshold's value when it first runs.

Nothing is read back to the host inside the loop: the live count stays on
the device, every launch is sized to the capacity, and the caller reads the
status word when it wants to.  Two drivers share the buffers:
  step_autograd()  one iteration through torch.autograd (GaussianRenderL1,
                   loss.backward(), then the library's SGD step)
  run(iters)       replays a CUDA graph of the iteration and one of the event
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib as L
from .api import LAS_PAPER, Renderer, _ptr, _stream_handle, edge_map, las_params, lib, new_status
from .autograd import GaussianRenderL1

GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")


class DensifyLoop:
    def __init__(self, gs, cams, targets, lr: float = 1e-3, every: int = 20, k_event: int = 50_000,
                 las: dict = LAS_PAPER, pair_capacity: int = 1 << 26, variants=(0, 0), device="cuda",
                 grad_threshold: float | None = None, warmup_events: int = 3, selection: str = "topk",
                 schedule: dict | None = None, densify_from: int = 0, densify_until: int | None = None,
                 budget: int = 0):
        """schedule: {"steps": T, group: (lr_init, lr_final), ...} exponential
        learning-rate decay per group on the device (Sec. 2.3; groups not named
        keep lr); densify_from / densify_until: the iterations between which the
        events run (the paper: every 500 in [500, 15000]); budget: Gaussians
        never exceed it (the split count is capped on the device)."""
        if selection not in ("topk", "sample"):
            raise ValueError("selection: 'topk' or 'sample'")
        if selection == "sample" and grad_threshold is not None:
            raise ValueError("the gradient threshold gates the top-k selection only")
        self.selection = selection
        self.gs, self.lr, self.every, self.k_event = gs, float(lr), int(every), int(k_event)
        self.grad_threshold = None if grad_threshold is None else float(grad_threshold)
        self.warmup_events = int(warmup_events)
        self.events = 0
        self.device = device
        self.targets = list(targets)
        self.status = new_status(device)
        self.E, self.medians, _, _ = edge_map(self.targets, status=self.status)
        self.r = Renderer(gs, cams, pair_capacity, device=device, variants=variants)
        cap = gs.capacity
        self.score = torch.zeros(cap, device=device)
        self.expv = torch.empty(cap, device=device) if selection == "sample" else None
        self.pos_grad = None
        if self.grad_threshold is not None:
            self.pos_grad = (torch.zeros(cap, device=device), torch.zeros(cap, dtype=torch.int32, device=device))
        self.grads = {k: torch.zeros_like(getattr(gs, k)) for k in GROUPS}
        npix = self.r.total_pix
        self.bufs = {"rgb": torch.empty((npix, 3), device=device), "T": torch.empty(npix, device=device),
                     "last": torch.empty(npix, dtype=torch.int32, device=device),
                     "loss": torch.empty(1, device=device)}
        self.mask = torch.zeros(cap, dtype=torch.uint8, device=device)
        self.selected = torch.zeros(1, dtype=torch.int32, device=device)
        self.ws_las = torch.empty(max(int(lib().gsp_las_workspace_size(cap)), 1), dtype=torch.uint8, device=device)
        self.las = las_params(las)
        self.densify_from, self.densify_until, self.budget = int(densify_from), densify_until, int(budget)
        self.sched = None
        if schedule is not None:
            rates = [tuple(schedule.get(k, (self.lr, self.lr))) for k in GROUPS]
            self.sched = L.LrSchedule((L.c_f32 * 5)(*[r[0] for r in rates]), (L.c_f32 * 5)(*[r[1] for r in rates]),
                                      int(schedule["steps"]))
        self.step_dev = torch.zeros(1, dtype=torch.int32, device=device)  # the schedule's step
        self.iteration_count = 0
        self._graphs = None

    # ---------------------------------------------------------- pieces
    def _sgd(self, grads, stream=None):
        if self.sched is not None:
            L.check(lib().gsp_sgd_step_scheduled(ctypes.byref(self.gs.struct()), *[_ptr(grads[k]) for k in GROUPS],
                                                 ctypes.byref(self.sched), _ptr(self.step_dev),
                                                 _stream_handle(stream)), "gsp_sgd_step_scheduled")
            return
        L.check(lib().gsp_sgd_step(ctypes.byref(self.gs.struct()), *[_ptr(grads[k]) for k in GROUPS],
                                   ctypes.c_float(self.lr), _stream_handle(stream)), "gsp_sgd_step")

    def event_due(self, iteration: int) -> bool:
        """Whether an event follows iteration `iteration` (1-based)."""
        return (iteration % self.every == 0 and iteration >= self.densify_from and
                (self.densify_until is None or iteration <= self.densify_until))

    def iteration(self, stream=None):
        """Forward + L1 + adjoint with fused edge score + SGD (library calls only)."""
        out = self.r.forward(targets=self.targets, status=self.status, out=self.bufs, stream=stream)
        self.r.backward(out, targets=self.targets, edge=self.E, score=self.score, grads=self.grads,
                        status=self.status, stream=stream, pos_grad=self.pos_grad)
        self._sgd(self.grads, stream)

    def gated(self) -> bool:
        """Whether the next event applies the gradient-threshold masking."""
        return self.pos_grad is not None and self.events >= self.warmup_events

    def event(self, stream=None, gated=None, count: bool = True):
        """Top-k by edge score (among the gradient-threshold candidates once the
        warm-up is over), Long-Axis-Split, score and statistic reset.  count:
        advance the event counter (not while the event is being captured)."""
        cap = self.gs.capacity
        s = _stream_handle(stream)
        if gated is None:
            gated = self.gated()
        expv = None
        if self.selection == "sample":
            # fresh Exp(1) variates (inputs of the sampling), drawn on the stream
            with torch.cuda.stream(stream) if stream is not None else torch.cuda.stream(
                    torch.cuda.current_stream(self.device)):
                self.expv.exponential_()
            expv = _ptr(self.expv).value
        pg = self.pos_grad if gated else None
        opts = L.SelectOpts(_ptr(pg[0]).value if pg else None, _ptr(pg[1]).value if pg else None,
                            float(self.grad_threshold or 0.0), expv, self.budget)
        L.check(lib().gsp_select_mask(_ptr(self.score), _ptr(self.gs.count), cap, self.k_event, ctypes.byref(opts),
                                      _ptr(self.mask), _ptr(self.selected), _ptr(self.ws_las), self.ws_las.numel(),
                                      _ptr(self.status), s), "gsp_select_mask")
        L.check(lib().gsp_las_split(ctypes.byref(self.gs.struct()), _ptr(self.mask), None, 0,
                                    ctypes.byref(self.las), _ptr(self.ws_las), self.ws_las.numel(),
                                    _ptr(self.status), s), "gsp_las_split")
        self.score.zero_()
        if self.pos_grad is not None:
            self.pos_grad[0].zero_()
            self.pos_grad[1].zero_()
        if count:
            self.events += 1

    def step_autograd(self):
        """One iteration through torch.autograd; the event follows every `every` iterations."""
        params = [getattr(self.gs, k) for k in GROUPS]
        for p in params:
            p.requires_grad_(True)
        loss = GaussianRenderL1.apply(*params, self.r, self.targets, self.E, self.score, self.pos_grad)
        loss.backward()
        with torch.no_grad():
            self._sgd({k: p.grad for k, p in zip(GROUPS, params)})
        for p in params:
            p.grad = None
            p.requires_grad_(False)
        self.iteration_count += 1
        if self.event_due(self.iteration_count):
            self.event()
        return loss.detach()

    # ---------------------------------------------------------- graphs
    def capture(self):
        """CUDA graphs of one iteration and of the events (warm-up and, with a
        gradient threshold, gated; capacity-sized launches, device-resident
        count: valid for every later state)."""
        side = torch.cuda.Stream(device=self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        g_it, g_ev = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        g_gated = torch.cuda.CUDAGraph() if self.pos_grad is not None else None
        with torch.cuda.stream(side):
            with torch.cuda.graph(g_it, stream=side):
                self.iteration(stream=side)
            with torch.cuda.graph(g_ev, stream=side):
                self.event(stream=side, gated=False, count=False)
            if g_gated is not None:
                with torch.cuda.graph(g_gated, stream=side):
                    self.event(stream=side, gated=True, count=False)
        torch.cuda.current_stream(self.device).wait_stream(side)
        self._graphs = (g_it, g_ev, g_gated)

    def run(self, iterations: int):
        """Replay `iterations` iterations (events included) without host reads."""
        if self._graphs is None:
            self.capture()
        g_it, g_ev, g_gated = self._graphs
        for _ in range(iterations):
            g_it.replay()
            self.iteration_count += 1
            if self.event_due(self.iteration_count):
                (g_gated if self.gated() else g_ev).replay()
                self.events += 1

    def loss(self) -> torch.Tensor:
        return self.bufs["loss"]
