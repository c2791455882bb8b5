"""Device-resident densification loop around the edge-guided densification.

One iteration: splatting forward over the fixed views with the L1 loss, the
adjoint with the edge score (Sec. 1, "Edge-Score importance") accumulated in
the same pass, and a plain SGD step on every parameter.  Every `every`
iterations a densification event takes the top-k Gaussians by accumulated
edge score, splits them with the Long-Axis-Split (Sec. 2.2, Alg. 1-2) into
the free capacity rows, and clears the scores.  The edge maps of the fixed
target views (Sec. 2.1) are computed once, in one fused launch.

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
from .api import LAS_CONFIG, Renderer, _ptr, _stream_handle, edge_map, las_params, lib, new_status
from .autograd import GaussianRenderL1

GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")


class DensifyLoop:
    def __init__(self, gs, cams, targets, lr: float = 1e-3, every: int = 20, k_event: int = 50_000,
                 las: dict = LAS_CONFIG, pair_capacity: int = 1 << 26, variants=(0, 0), device="cuda"):
        self.gs, self.lr, self.every, self.k_event = gs, float(lr), int(every), int(k_event)
        self.device = device
        self.targets = list(targets)
        self.status = new_status(device)
        self.E, self.medians, _, _ = edge_map(self.targets, status=self.status)
        self.r = Renderer(gs, cams, pair_capacity, device=device, variants=variants)
        cap = gs.capacity
        self.score = torch.zeros(cap, device=device)
        self.grads = {k: torch.zeros_like(getattr(gs, k)) for k in GROUPS}
        npix = self.r.total_pix
        self.bufs = {"rgb": torch.empty((npix, 3), device=device), "T": torch.empty(npix, device=device),
                     "last": torch.empty(npix, dtype=torch.int32, device=device),
                     "loss": torch.empty(1, device=device)}
        self.mask = torch.zeros(cap, dtype=torch.uint8, device=device)
        self.selected = torch.zeros(1, dtype=torch.int32, device=device)
        self.ws_las = torch.empty(max(int(lib().gsp_las_workspace_size(cap)), 1), dtype=torch.uint8, device=device)
        self.las = las_params(las)
        self.iteration_count = 0
        self._graphs = None

    # ---------------------------------------------------------- pieces
    def _sgd(self, grads, stream=None):
        L.check(lib().gsp_sgd_step(ctypes.byref(self.gs.struct()), *[_ptr(grads[k]) for k in GROUPS],
                                   ctypes.c_float(self.lr), _stream_handle(stream)), "gsp_sgd_step")

    def iteration(self, stream=None):
        """Forward + L1 + adjoint with fused edge score + SGD (library calls only)."""
        out = self.r.forward(targets=self.targets, status=self.status, out=self.bufs, stream=stream)
        self.r.backward(out, targets=self.targets, edge=self.E, score=self.score, grads=self.grads,
                        status=self.status, stream=stream)
        self._sgd(self.grads, stream)

    def event(self, stream=None):
        """Top-k by edge score, Long-Axis-Split, score reset."""
        cap = self.gs.capacity
        s = _stream_handle(stream)
        L.check(lib().gsp_topk_mask(_ptr(self.score), _ptr(self.gs.count), cap, self.k_event, _ptr(self.mask),
                                    _ptr(self.selected), _ptr(self.ws_las), self.ws_las.numel(), _ptr(self.status),
                                    s), "gsp_topk_mask")
        L.check(lib().gsp_las_split(ctypes.byref(self.gs.struct()), _ptr(self.mask), None, 0,
                                    ctypes.byref(self.las), _ptr(self.ws_las), self.ws_las.numel(),
                                    _ptr(self.status), s), "gsp_las_split")
        self.score.zero_()

    def step_autograd(self):
        """One iteration through torch.autograd; the event follows every `every` iterations."""
        params = [getattr(self.gs, k) for k in GROUPS]
        for p in params:
            p.requires_grad_(True)
        loss = GaussianRenderL1.apply(*params, self.r, self.targets, self.E, self.score)
        loss.backward()
        with torch.no_grad():
            self._sgd({k: p.grad for k, p in zip(GROUPS, params)})
        for p in params:
            p.grad = None
            p.requires_grad_(False)
        self.iteration_count += 1
        if self.iteration_count % self.every == 0:
            self.event()
        return loss.detach()

    # ---------------------------------------------------------- graphs
    def capture(self):
        """CUDA graphs of one iteration and of one event (capacity-sized launches,
        device-resident count: valid for every later state)."""
        side = torch.cuda.Stream(device=self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        g_it, g_ev = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            with torch.cuda.graph(g_it, stream=side):
                self.iteration(stream=side)
            with torch.cuda.graph(g_ev, stream=side):
                self.event(stream=side)
        torch.cuda.current_stream(self.device).wait_stream(side)
        self._graphs = (g_it, g_ev)

    def run(self, iterations: int):
        """Replay `iterations` iterations (events included) without host reads."""
        if self._graphs is None:
            self.capture()
        g_it, g_ev = self._graphs
        for _ in range(iterations):
            g_it.replay()
            self.iteration_count += 1
            if self.iteration_count % self.every == 0:
                g_ev.replay()

    def loss(self) -> torch.Tensor:
        return self.bufs["loss"]
