"""Torch-facing wrappers of the libgsp entry points (argument marshalling only).

Every function hands device pointers of CUDA tensors and the current CUDA
stream to the C ABI; all arithmetic runs in the library's kernels.  PyTorch
supplies device memory and streams.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from . import _lib as L

LAS_PAPER = {"k_off": 0.5, "long_factor": 0.5, "other_factor": 0.85, "beta": 0.6}
LAS_CONFIG = {"k_off": 1.0, "long_factor": 0.5, "other_factor": 1.0, "beta": 0.6}


def lib():
    return L.load()


def _stream_handle(stream=None) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t) -> ctypes.c_void_p | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    return ctypes.c_void_p(t.data_ptr())


def _event_handle(ev) -> int | None:
    """The cudaEvent_t of a torch.cuda.Event (created on the current stream if it
    has not been yet), or None."""
    if ev is None:
        return None
    if not ev.cuda_event:
        ev.record()
    return int(ev.cuda_event)


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def new_status(device="cuda") -> torch.Tensor:
    return torch.zeros(1, dtype=torch.int32, device=device)


def raise_on_device_status(status: torch.Tensor, where: str = "device"):
    """Synchronising read of a device status word; raises GspError if set."""
    L.check(int(status.item()), where)


def image_desc(img: torch.Tensor, out_offset: int = 0) -> L.ImageDesc:
    """Descriptor of an HWC uint8 CUDA image; rows may be padded (row pitch = stride(0))."""
    if img.dtype != torch.uint8 or img.dim() != 3 or img.shape[2] != 3:
        raise ValueError("uint8 [H, W, 3] image expected")
    if img.stride(2) != 1 or img.stride(1) != 3:
        raise ValueError("pixels must be packed RGB (row padding allowed)")
    h, w = int(img.shape[0]), int(img.shape[1])
    return L.ImageDesc(img.data_ptr(), w, h, int(img.stride(0)), int(out_offset))


def pitched_image(img: torch.Tensor, align: int = 16) -> torch.Tensor:
    """Copy an HWC uint8 image into rows padded to a multiple of `align` bytes."""
    h, w = int(img.shape[0]), int(img.shape[1])
    pitch = (3 * w + align - 1) // align * align
    buf = torch.empty((h, pitch), dtype=torch.uint8, device=img.device)
    view = buf[:, :3 * w].view(h, w, 3)
    view.copy_(img)
    return view


# ----------------------------------------------------------------- edge map

def edge_map(images, *, mode: str = "fused", taps=None, sigma: float = 1.0, with_mask: bool = False,
             spin_limit: int = 0, test_expire: int = 0, blocks_per_sm: int = 0, out: torch.Tensor | None = None,
             status: torch.Tensor | None = None, workspace: torch.Tensor | None = None, stream=None):
    """Edge-importance maps of a list of HWC uint8 CUDA views (one launch in fused mode).

    Returns (E, medians, mask, status): E is a flat float32 tensor holding the
    views one after another (row-major), medians is [V], mask is uint8 like E
    (or None), status is the device status word.  spin_limit and test_expire
    are gsp_edge_opts' bounded-wait limit and failure-injection hook (tests);
    blocks_per_sm caps the fused launch's blocks per SM (0: as many as fit).
    """
    if isinstance(images, torch.Tensor):
        images = [images]
    v = len(images)
    descs = (L.ImageDesc * v)()
    off = 0
    for i, img in enumerate(images):
        descs[i] = image_desc(img, off)
        off += int(img.shape[0]) * int(img.shape[1])
    dev = images[0].device
    opts = L.EdgeOpts()
    lib().gsp_edge_opts_default(ctypes.byref(opts))
    opts.mode = L.GSP_EDGE_FUSED if mode == "fused" else L.GSP_EDGE_PLAIN
    if taps is not None:
        opts.use_custom_taps = 1
        for k in range(5):
            opts.taps[k] = float(taps[k])
    opts.sigma = float(sigma)
    opts.spin_limit = int(spin_limit)
    opts.test_expire = int(test_expire)
    opts.blocks_per_sm = int(blocks_per_sm)
    need = lib().gsp_edge_map_workspace_size(descs, v, ctypes.byref(opts))
    if need == 0:
        raise L.GspError(L.GSP_ERR_INVALID_ARG, "gsp_edge_map_workspace_size")
    ws = workspace if workspace is not None and workspace.numel() >= need else _workspace(need, dev)
    E = out if out is not None else torch.empty(off, dtype=torch.float32, device=dev)
    med = torch.empty(v, dtype=torch.float32, device=dev)
    mask = torch.empty(off, dtype=torch.uint8, device=dev) if with_mask else None
    st = status if status is not None else new_status(dev)
    L.check(lib().gsp_edge_map(descs, v, _ptr(E), _ptr(med), _ptr(mask), ctypes.byref(opts), _ptr(ws), need,
                               _ptr(st), _stream_handle(stream)), "gsp_edge_map")
    return E, med, mask, st


# ---------------------------------------------------------------- splatting

@dataclass
class GaussianSet:
    """Caller-owned parameter storage with `capacity` rows and a device count."""
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    opacity_logits: torch.Tensor
    sh: torch.Tensor
    count: torch.Tensor
    sh_degree: int

    @property
    def capacity(self) -> int:
        return int(self.means.shape[0])

    @property
    def K(self) -> int:
        return (self.sh_degree + 1) ** 2

    @staticmethod
    def from_arrays(arrs: dict, capacity: int | None = None, device="cuda") -> "GaussianSet":
        n = int(arrs["means"].shape[0])
        cap = max(capacity or n, 1)
        k = (int(arrs["sh_degree"]) + 1) ** 2

        def put(name, shape):
            t = torch.zeros((cap,) + shape, dtype=torch.float32, device=device)
            if n:
                t[:n] = torch.as_tensor(arrs[name], dtype=torch.float32).reshape((n,) + shape).to(device)
            return t

        return GaussianSet(put("means", (3,)), put("log_scales", (3,)), put("quats", (4,)),
                           put("opacity_logits", ()), put("sh", (k, 3)),
                           torch.tensor([n], dtype=torch.int32, device=device), int(arrs["sh_degree"]))

    def struct(self) -> L.Gaussians:
        for t in (self.means, self.log_scales, self.quats, self.opacity_logits, self.sh):
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
                raise ValueError("parameters must be contiguous float32 CUDA tensors")
        return L.Gaussians(self.means.data_ptr(), self.log_scales.data_ptr(), self.quats.data_ptr(),
                           self.opacity_logits.data_ptr(), self.sh.data_ptr(), self.count.data_ptr(),
                           self.capacity, self.sh_degree)


def camera_struct(cam: dict, pixel_offset: int = 0) -> L.Camera:
    c = L.Camera()
    vm = [float(x) for x in torch.as_tensor(cam["viewmat"], dtype=torch.float32).reshape(12).tolist()]
    for k in range(12):
        c.viewmat[k] = vm[k]
    c.fx, c.fy, c.cx, c.cy = float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"])
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.pixel_offset = int(pixel_offset)
    return c


class Renderer:
    """Workspace and camera set of one gsp_render_fwd / gsp_render_bwd pairing."""

    def __init__(self, gs: GaussianSet, cams: list, pair_capacity: int, device="cuda",
                 workspace: torch.Tensor | None = None, variants: tuple[int, int] = (0, 0)):
        self.gs = gs
        self.nv = len(cams)
        self.cams = (L.Camera * self.nv)()
        off = 0
        self.offsets = []
        for i, c in enumerate(cams):
            self.cams[i] = camera_struct(c, off)
            self.offsets.append(off)
            off += int(c["width"]) * int(c["height"])
        self.total_pix = off
        self.opts = L.RenderOpts(int(pair_capacity), int(variants[0]), int(variants[1]))
        # gsp_render_opts.spin_limit / test_expire: the depth sort's look-back limit and
        # the failure-injection hook (tests); 0 in normal use
        self.spin_limit = 0
        self.test_expire = 0
        # gsp_render_opts.list_prefix: tile-list entries written before the forward
        # compositing (0: the library's default; results do not depend on it)
        self.list_prefix = 0
        # pixels of the whole L1 loss when it spans views rendered elsewhere (0: these views)
        self.loss_pixels = 0
        self.ws_bytes = lib().gsp_render_workspace_size(gs.capacity, gs.sh_degree, self.cams, self.nv,
                                                        ctypes.byref(self.opts))
        if self.ws_bytes == 0:
            raise L.GspError(L.GSP_ERR_INVALID_ARG, "gsp_render_workspace_size")
        if workspace is not None and workspace.numel() >= self.ws_bytes:
            self.ws = workspace
        else:
            self.ws = _workspace(self.ws_bytes, device)
        self.device = device

    @property
    def variants(self) -> tuple[int, int]:
        return int(self.opts.fwd_variant), int(self.opts.bwd_variant)

    @variants.setter
    def variants(self, v: tuple[int, int]):
        self.opts.fwd_variant, self.opts.bwd_variant = int(v[0]), int(v[1])

    def stats(self) -> torch.Tensor:
        """Device int64[3] of the last forward: tile-Gaussian pairs, composited pairs,
        tiles whose compositing went on past their list prefix."""
        p = lib().gsp_render_pair_count_ptr(_ptr(self.ws), self.gs.capacity, self.gs.sh_degree, self.cams,
                                            self.nv, ctypes.byref(self.opts))
        off = int(p) - self.ws.data_ptr()
        return self.ws[off:off + 24].view(torch.int64)

    def pair_count(self) -> torch.Tensor:
        return self.stats()[0:1]

    def _targets(self, targets):
        if targets is None:
            return None
        arr = (L.ImageDesc * self.nv)()
        for i, t in enumerate(targets):
            arr[i] = image_desc(t, 0)
        return arr

    def _opts(self, pos_grad=None, score_event=None) -> L.RenderOpts:
        o = self.opts
        return L.RenderOpts(o.pair_capacity, o.fwd_variant, o.bwd_variant,
                            _ptr(pos_grad[0]).value if pos_grad is not None else None,
                            _ptr(pos_grad[1]).value if pos_grad is not None else None,
                            int(self.loss_pixels), int(self.spin_limit), int(self.test_expire),
                            _event_handle(score_event), int(self.list_prefix))

    def forward(self, targets=None, edge=None, score=None, want_loss: bool = True, status=None, stream=None,
                out=None):
        dev = self.device
        o = out or {}
        rgb = o.get("rgb") if o.get("rgb") is not None else torch.empty((self.total_pix, 3), dtype=torch.float32,
                                                                           device=dev)
        T = o.get("T") if o.get("T") is not None else torch.empty(self.total_pix, dtype=torch.float32, device=dev)
        last = o.get("last") if o.get("last") is not None else torch.empty(self.total_pix, dtype=torch.int32,
                                                                            device=dev)
        loss = None
        if targets is not None and want_loss:
            loss = o.get("loss") if o.get("loss") is not None else torch.empty(1, dtype=torch.float32, device=dev)
        st = status if status is not None else new_status(dev)
        L.check(lib().gsp_render_fwd(ctypes.byref(self.gs.struct()), self.cams, self.nv, self._targets(targets),
                                     _ptr(edge), _ptr(rgb), _ptr(T), _ptr(last), _ptr(score), _ptr(loss),
                                     ctypes.byref(self._opts()), _ptr(self.ws), self.ws_bytes, _ptr(st),
                                     _stream_handle(stream)), "gsp_render_fwd")
        return {"rgb": rgb, "T": T, "last": last, "loss": loss, "status": st}

    def backward(self, fwd: dict, targets=None, dL_drgb=None, edge=None, score=None, grads=None,
                 accumulate: bool = False, status=None, stream=None, pos_grad=None, score_event=None):
        """pos_grad: optional (sum float32 [capacity], count int32 [capacity]) device
        tensors; the positional statistic of the gradient-threshold masking is
        added to them (see gsp_render_opts).  score_event: optional
        torch.cuda.Event, recorded once the edge score is complete (before the
        chain to the parameters has finished)."""
        gs = self.gs
        opts = self._opts(pos_grad, score_event)
        if grads is None:
            grads = {"means": torch.zeros_like(gs.means), "log_scales": torch.zeros_like(gs.log_scales),
                     "quats": torch.zeros_like(gs.quats), "opacity_logits": torch.zeros_like(gs.opacity_logits),
                     "sh": torch.zeros_like(gs.sh)}
        st = status if status is not None else fwd.get("status", new_status(self.device))
        L.check(lib().gsp_render_bwd(ctypes.byref(gs.struct()), self.cams, self.nv, self._targets(targets),
                                     _ptr(dL_drgb), _ptr(fwd["rgb"]), _ptr(fwd["T"]), _ptr(fwd["last"]), _ptr(edge),
                                     _ptr(score), _ptr(grads["means"]), _ptr(grads["log_scales"]),
                                     _ptr(grads["quats"]), _ptr(grads["opacity_logits"]), _ptr(grads["sh"]),
                                     int(bool(accumulate)), ctypes.byref(opts), _ptr(self.ws), self.ws_bytes,
                                     _ptr(st), _stream_handle(stream)), "gsp_render_bwd")
        return grads


# ------------------------------------------------------ selection and split

def las_params(p: dict) -> L.LasParams:
    return L.LasParams(float(p["k_off"]), float(p["long_factor"]), float(p["other_factor"]), float(p["beta"]))


def topk_mask(scores: torch.Tensor, count: torch.Tensor, k: int, status=None, stream=None):
    cap = int(scores.shape[0])
    need = lib().gsp_las_workspace_size(cap)
    ws = _workspace(need, scores.device)
    mask = torch.empty(cap, dtype=torch.uint8, device=scores.device)
    sel = torch.zeros(1, dtype=torch.int32, device=scores.device)
    st = status if status is not None else new_status(scores.device)
    L.check(lib().gsp_topk_mask(_ptr(scores), _ptr(count), cap, int(k), _ptr(mask), _ptr(sel), _ptr(ws), need,
                                _ptr(st), _stream_handle(stream)), "gsp_topk_mask")
    return mask, sel, st


def topk_mask_gated(scores: torch.Tensor, pos_grad_sum: torch.Tensor, pos_grad_count: torch.Tensor,
                    threshold: float, count: torch.Tensor, k: int, status=None, stream=None):
    """Top-k among the Gaussians whose mean positional gradient reaches threshold
    (gradient-threshold masking, gsp_topk_mask_gated)."""
    cap = int(scores.shape[0])
    need = lib().gsp_las_workspace_size(cap)
    ws = _workspace(need, scores.device)
    mask = torch.empty(cap, dtype=torch.uint8, device=scores.device)
    sel = torch.zeros(1, dtype=torch.int32, device=scores.device)
    st = status if status is not None else new_status(scores.device)
    L.check(lib().gsp_topk_mask_gated(_ptr(scores), _ptr(pos_grad_sum), _ptr(pos_grad_count),
                                      ctypes.c_float(threshold), _ptr(count), cap, int(k), _ptr(mask), _ptr(sel),
                                      _ptr(ws), need, _ptr(st), _stream_handle(stream)), "gsp_topk_mask_gated")
    return mask, sel, st


def sample_mask(scores: torch.Tensor, exp_variates: torch.Tensor, count: torch.Tensor, k: int, status=None,
                stream=None):
    """Importance sampling of k Gaussians by edge score (gsp_sample_mask);
    exp_variates: Exp(1) draws, one per row (e.g. torch.empty_like(scores).exponential_())."""
    cap = int(scores.shape[0])
    need = lib().gsp_las_workspace_size(cap)
    ws = _workspace(need, scores.device)
    mask = torch.empty(cap, dtype=torch.uint8, device=scores.device)
    sel = torch.zeros(1, dtype=torch.int32, device=scores.device)
    st = status if status is not None else new_status(scores.device)
    L.check(lib().gsp_sample_mask(_ptr(scores), _ptr(exp_variates), _ptr(count), cap, int(k), _ptr(mask), _ptr(sel),
                                  _ptr(ws), need, _ptr(st), _stream_handle(stream)), "gsp_sample_mask")
    return mask, sel, st


def select_mask(scores: torch.Tensor, count: torch.Tensor, k: int, pos_grad=None, threshold: float = 0.0,
                exp_variates=None, budget: int = 0, status=None, stream=None, workspace=None, out=None):
    """gsp_select_mask: top-k or importance sampling, optionally gated by the
    gradient threshold (pos_grad = (sum, count)) and capped by a Gaussian budget."""
    cap = int(scores.shape[0])
    need = lib().gsp_las_workspace_size(cap)
    ws = workspace if workspace is not None else _workspace(need, scores.device)
    mask = out if out is not None else torch.empty(cap, dtype=torch.uint8, device=scores.device)
    sel = torch.zeros(1, dtype=torch.int32, device=scores.device)
    st = status if status is not None else new_status(scores.device)
    o = L.SelectOpts(_ptr(pos_grad[0]).value if pos_grad is not None else None,
                     _ptr(pos_grad[1]).value if pos_grad is not None else None, float(threshold),
                     _ptr(exp_variates).value if exp_variates is not None else None, int(budget), 0, 0)
    L.check(lib().gsp_select_mask(_ptr(scores), _ptr(count), cap, int(k), ctypes.byref(o), _ptr(mask), _ptr(sel),
                                  _ptr(ws), ws.numel(), _ptr(st), _stream_handle(stream)), "gsp_select_mask")
    return mask, sel, st


def launch_count() -> int:
    """Kernels and memsets the library has enqueued in this process."""
    return int(lib().gsp_kernel_launch_count())


class StageTimer:
    """Library-recorded CUDA events around every occurrence of one stage."""

    def __init__(self, stage: str, max_records: int = 1024):
        L.check(lib().gsp_stage_timer_arm(stage.encode(), int(max_records)), "gsp_stage_timer_arm")
        self.stage = stage

    def read(self):
        ms, n = ctypes.c_float(0.0), ctypes.c_int32(0)
        L.check(lib().gsp_stage_timer_read(ctypes.byref(ms), ctypes.byref(n)), "gsp_stage_timer_read")
        return float(ms.value), int(n.value)

    @staticmethod
    def disarm():
        L.check(lib().gsp_stage_timer_arm(None, 0), "gsp_stage_timer_arm")


def las_split(gs: GaussianSet, mask: torch.Tensor | None = None, scores: torch.Tensor | None = None, k: int = 0,
              params: dict = LAS_CONFIG, status=None, workspace=None, stream=None):
    need = lib().gsp_las_workspace_size(gs.capacity)
    ws = workspace if workspace is not None and workspace.numel() >= need else _workspace(need, gs.means.device)
    st = status if status is not None else new_status(gs.means.device)
    p = las_params(params)
    L.check(lib().gsp_las_split(ctypes.byref(gs.struct()), _ptr(mask), _ptr(scores), int(k), ctypes.byref(p),
                                _ptr(ws), need, _ptr(st), _stream_handle(stream)), "gsp_las_split")
    return st
