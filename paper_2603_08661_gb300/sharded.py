"""View-sharded data parallelism: one process per GPU, the views split over the ranks.

The edge-guided densification path shards over views.  Every rank holds the
whole Gaussian set and renders only the views assigned to it: forward with the
L1 loss and the edge score (Sec. 1, "Edge-Score importance"), then the adjoint.
Per-Gaussian gradients and scores are sums over views, so one all-reduce (sum)
of one flat buffer - the gradients of every parameter group (59 floats per
Gaussian at SH degree 3), the edge score (1 float) and the loss (1 float) -
gives every rank the result of the whole view set.  What follows (the SGD
step, the top-k selection and the Long-Axis-Split of Sec. 2.2) is
deterministic and runs replicated on every rank, so the parameter sets stay
identical without any further exchange.

The loss is a mean over the pixels of all views on all ranks: each rank's
adjoint is normalised by that global pixel count (gsp_render_opts.loss_pixels),
so the per-rank results sum to the whole loss and its gradient.

The all-reduce is torch.distributed's: NCCL sums the device buffer in place;
with gloo (CPU tests, or ranks that share one GPU) the buffer is summed through
host memory.  No kernel of one rank ever waits on another rank.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from .api import Renderer

GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def partition_views(pixels, world: int) -> list[list[int]]:
    """Balanced, deterministic assignment of views to ranks by pixel count.

    Views are taken in descending pixel count (ties by ascending index) and each
    goes to the rank with the fewest pixels so far (ties to the lower rank); the
    views of a rank are returned in ascending index order.  A rank may get no
    view when there are fewer views than ranks."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for v in sorted(range(len(pixels)), key=lambda i: (-int(pixels[i]), i)):
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(v)
        load[r] += int(pixels[v])
    return [sorted(p) for p in parts]


class FlatGrads:
    """One contiguous float32 buffer: the gradient of every parameter group, the
    edge score and the loss - the unit of the all-reduce.  The named tensors are
    views into it, shaped like the parameters."""

    def __init__(self, capacity: int, sh_degree: int, device="cuda"):
        k = (int(sh_degree) + 1) ** 2
        self.capacity, self.sh_degree = int(capacity), int(sh_degree)
        shapes = {"means": (3,), "log_scales": (3,), "quats": (4,), "opacity_logits": (), "sh": (k, 3),
                  "score": ()}
        sizes = {n: self.capacity * (1 if not s else int(torch.tensor(s).prod())) for n, s in shapes.items()}
        total = sum(sizes.values()) + 1
        self.flat = torch.zeros(total, dtype=torch.float32, device=device)
        off = 0
        self.views = {}
        for n, s in shapes.items():
            self.views[n] = self.flat[off:off + sizes[n]].view((self.capacity,) + s)
            off += sizes[n]
        self.views["loss"] = self.flat[off:off + 1]

    def __getitem__(self, name: str) -> torch.Tensor:
        return self.views[name]

    @property
    def grads(self) -> dict:
        return {n: self.views[n] for n in GROUPS}

    def zero_(self):
        self.flat.zero_()


def all_reduce_flat(flat: torch.Tensor, group=None) -> torch.Tensor:
    """Sum `flat` over the ranks of `group`, in place.  NCCL reduces device
    memory directly; any other backend (gloo) gets a host copy, reduced and
    copied back."""
    if dist.get_backend(group) == "nccl" or not flat.is_cuda:
        dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
        return flat
    host = flat.cpu()
    dist.all_reduce(host, op=dist.ReduceOp.SUM, group=group)
    flat.copy_(host)
    return flat


class ShardedRenderer:
    """Forward + L1 loss + edge score + adjoint over this rank's share of the views,
    then one all-reduce.  cams / targets / edges are the whole view set (the same
    list on every rank); `views` is this rank's share (partition_views)."""

    def __init__(self, gs, cams: list, pair_capacity: int, group=None, device="cuda", variants=(0, 0),
                 rank: int | None = None, world: int | None = None):
        self.gs, self.group, self.device = gs, group, device
        self.rank = dist.get_rank(group) if rank is None else int(rank)
        self.world = dist.get_world_size(group) if world is None else int(world)
        pixels = [int(c["width"]) * int(c["height"]) for c in cams]
        self.total_pix = sum(pixels)
        self.offsets = [sum(pixels[:v]) for v in range(len(cams))]
        self.views = partition_views(pixels, self.world)[self.rank]
        self.r = None
        if self.views:
            self.r = Renderer(gs, [cams[v] for v in self.views], pair_capacity, device=device, variants=variants)
            self.r.loss_pixels = self.total_pix
        self.out = FlatGrads(gs.capacity, gs.sh_degree, device)

    def local_edge(self, edge: torch.Tensor | None) -> torch.Tensor | None:
        """This rank's views of a whole-view-set per-pixel map, concatenated."""
        if edge is None or not self.views:
            return None
        parts = [edge[self.offsets[v]:self.offsets[v] + self._pix(v)] for v in self.views]
        return torch.cat(parts) if len(parts) > 1 else parts[0].contiguous()

    def _pix(self, v: int) -> int:
        nxt = self.offsets[v + 1] if v + 1 < len(self.offsets) else self.total_pix
        return nxt - self.offsets[v]

    def step(self, targets: list, edge: torch.Tensor | None = None, status=None) -> FlatGrads:
        """One sharded iteration; returns the all-reduced FlatGrads (identical on
        every rank): gradients, edge score (when edge is given) and L1 loss."""
        o = self.out
        o.zero_()
        if self.r is not None:
            tg = [targets[v] for v in self.views]
            e = self.local_edge(edge)
            fwd = self.r.forward(targets=tg, edge=e, score=o["score"] if e is not None else None, status=status,
                                 out={"loss": o["loss"]})
            self.r.backward(fwd, targets=tg, grads=o.grads, accumulate=True, status=fwd["status"])
            self.status = fwd["status"]
        all_reduce_flat(o.flat, self.group)
        return o
