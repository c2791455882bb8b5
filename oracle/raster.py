"""Python side of the FP64 splatting oracle (test infrastructure only).

Wraps oracle/raster.c (projection, tile-binned and brute-force compositing,
edge score, analytic adjoint) and adds the L1 photometric loss and the
central finite-difference check of the adjoint.  The conventions are listed
in the header of raster.c.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

PROJ_STRIDE = 24
(P_VALID, P_ZKEY, P_Z, P_MX, P_MY, P_COV_A, P_COV_B, P_COV_C, P_CON_A, P_CON_B, P_CON_C,
 P_OPAC, P_R, P_G, P_B, P_RAW_R, P_RAW_G, P_RAW_B, P_RADIUS, P_TX0, P_TY0, P_TX1, P_TY1,
 P_SPARE) = range(24)

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        i64, ci = ctypes.c_int64, ctypes.c_int
        _lib.orc_project.argtypes = [i64, _dp, _dp, _dp, _dp, _dp, ci, _fp, _dp, ci, ci, _dp]
        _lib.orc_render.argtypes = [i64, _dp, ci, ci, _dp, ci, ci, ci, ci, ci, _dp, _dp, _i32p,
                                    _i64p, _dp, _dp, _i64p, i64]
        _lib.orc_order.argtypes = [i64, _dp, _i64p]
        _lib.orc_order.restype = i64
        _lib.orc_gate_affected.argtypes = [i64, _i64p, _dp, i64, _i32p, ctypes.c_double,
                                           ctypes.POINTER(ctypes.c_uint8)]
        _lib.orc_render_bwd.argtypes = [i64, _dp, _dp, _dp, _dp, _dp, ci, _fp, _dp, ci, ci, _dp,
                                        _dp, _dp, _dp, _dp, _dp, _dp, _dp, ctypes.POINTER(ctypes.c_int), ci]
        _lib.orc_sh_basis.argtypes = [i64, _dp, _dp]
        _lib.orc_quat_to_rot.argtypes = [i64, _dp, _dp]
    return _lib


def _p(a, t=_dp):
    return a.ctypes.data_as(t) if a is not None else None


def _params64(g: dict):
    c = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    return (c(g["means"]), c(g["log_scales"]), c(g["quats"]), c(g["opacity_logits"]), c(g["sh"]))


def _cam(cam: dict):
    """The camera as the library receives it: the view matrix and the pinhole
    intrinsics are the FP32 numbers of its camera record (both sides then
    compute the same function of the same inputs; the arithmetic stays FP64)."""
    vm = np.ascontiguousarray(cam["viewmat"], dtype=np.float32).reshape(12)
    intr = np.array([cam["fx"], cam["fy"], cam["cx"], cam["cy"]], dtype=np.float32).astype(np.float64)
    return vm, intr, int(cam["width"]), int(cam["height"])


def sh_basis(dirs: np.ndarray) -> np.ndarray:
    d = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((d.shape[0], 16))
    lib().orc_sh_basis(d.shape[0], _p(d), _p(out))
    return out


def quat_to_rot(q: np.ndarray) -> np.ndarray:
    q = np.ascontiguousarray(q, dtype=np.float64).reshape(-1, 4)
    out = np.zeros((q.shape[0], 9))
    lib().orc_quat_to_rot(q.shape[0], _p(q), _p(out))
    return out.reshape(-1, 3, 3)


def project(g: dict, cam: dict) -> np.ndarray:
    """Projected records, one row of PROJ_STRIDE doubles per Gaussian."""
    m, s, q, o, sh = _params64(g)
    vm, intr, w, h = _cam(cam)
    n = m.shape[0]
    out = np.zeros((n, PROJ_STRIDE))
    lib().orc_project(n, _p(m), _p(s), _p(q), _p(o), _p(sh), int(g["sh_degree"]), _p(vm, _fp),
                      _p(intr), w, h, _p(out))
    return out


def order(proj: np.ndarray) -> np.ndarray:
    """The valid Gaussians in compositing order (ascending depth key, then index)."""
    out = np.zeros(proj.shape[0], dtype=np.int64)
    m = lib().orc_order(proj.shape[0], _p(np.ascontiguousarray(proj)), _p(out, _i64p))
    return out[:m]


def gate_affected(proj: np.ndarray, mask: np.ndarray, window: float, order_=None) -> np.ndarray:
    """Boolean array over the Gaussians: True where the result at a pixel of
    mask (H x W) moves when a gate decision at that pixel flips (see
    orc_gate_affected)."""
    o = order(proj) if order_ is None else np.ascontiguousarray(order_, dtype=np.int64)
    ys, xs = np.nonzero(mask)
    xy = np.ascontiguousarray(np.stack([xs, ys], axis=1), dtype=np.int32)
    mark = np.zeros(proj.shape[0], dtype=np.uint8)
    lib().orc_gate_affected(o.shape[0], _p(o, _i64p), _p(np.ascontiguousarray(proj)), xy.shape[0],
                            _p(xy, _i32p), float(window), _p(mark, ctypes.POINTER(ctypes.c_uint8)))
    return mark.astype(bool)


def render(g: dict, cam: dict, edge=None, brute: bool = False, region=None, proj=None, order=None) -> dict:
    """Composite the view (or the pixel region (x0, y0, x1, y1) of it).

    order (optional): the compositing order of the valid Gaussians of proj
    (as returned by order()), to skip the sort."""
    proj = project(g, cam) if proj is None else proj
    w, h = int(cam["width"]), int(cam["height"])
    n = proj.shape[0]
    x0, y0, x1, y1 = region if region is not None else (0, 0, w, h)
    rgb = np.zeros((h, w, 3))
    T = np.ones((h, w))
    nc = np.zeros((h, w), dtype=np.int32)
    last = np.full((h, w), -1, dtype=np.int64)
    gap = np.full((h, w), np.inf)
    score = np.zeros(n)
    e = None if edge is None else np.ascontiguousarray(edge, dtype=np.float64)
    o = None if order is None else np.ascontiguousarray(order, dtype=np.int64)
    lib().orc_render(n, _p(np.ascontiguousarray(proj)), w, h, _p(e), int(brute), x0, y0, x1, y1,
                     _p(rgb), _p(T), _p(nc, _i32p), _p(last, _i64p), _p(score), _p(gap),
                     _p(o, _i64p), 0 if o is None else o.shape[0])
    return {"rgb": rgb, "T": T, "ncontrib": nc, "last_id": last, "score": score,
            "gate_gap": gap, "proj": proj}


def render_bwd(g: dict, cam: dict, dLdC: np.ndarray, proj=None, region=None, magnitude: bool = False) -> dict:
    """Analytic adjoint: parameter gradients of sum(dLdC * C).

    region (x0, y0, x1, y1), optional: dLdC is taken as zero outside it.
    magnitude=True returns the magnitude adjoint instead: for every gradient
    entry, the sum of the absolute values of the terms the adjoint adds up
    (every factor by its absolute value, every difference as a sum).  It is
    the condition of each entry: a result computed from terms that each carry
    a relative error e is off by at most e times it."""
    m, s, q, o, sh = _params64(g)
    vm, intr, w, h = _cam(cam)
    proj = project(g, cam) if proj is None else proj
    n = m.shape[0]
    k = sh.shape[1]
    out = {"means": np.zeros((n, 3)), "log_scales": np.zeros((n, 3)), "quats": np.zeros((n, 4)),
           "opacity_logits": np.zeros(n), "sh": np.zeros((n, k, 3)), "g2d": np.zeros((n, 9))}
    d = np.ascontiguousarray(dLdC, dtype=np.float64)
    lib().orc_render_bwd(n, _p(m), _p(s), _p(q), _p(o), _p(sh), int(g["sh_degree"]), _p(vm, _fp),
                         _p(intr), w, h, _p(np.ascontiguousarray(proj)), _p(d), _p(out["means"]),
                         _p(out["log_scales"]), _p(out["quats"]), _p(out["opacity_logits"]),
                         _p(out["sh"]), _p(out["g2d"]),
                         None if region is None else (ctypes.c_int * 4)(*[int(r) for r in region]),
                         1 if magnitude else 0)
    return out


def l1_loss(rgb: np.ndarray, target_u8: np.ndarray):
    """Mean over H*W*3 of |C - target/255| and its gradient dL/dC (sign(0) = 0)."""
    t = target_u8.astype(np.float64) / 255.0
    diff = rgb - t
    return float(np.abs(diff).mean()), np.sign(diff) / diff.size


def _footprint(rec: np.ndarray, w: int, h: int):
    if rec[P_VALID] == 0 or rec[P_RADIUS] < 0:
        return None
    r = rec[P_RADIUS] + 1.0
    return (max(int(np.floor(rec[P_MX] - r)), 0), max(int(np.floor(rec[P_MY] - r)), 0),
            min(int(np.ceil(rec[P_MX] + r)) + 1, w), min(int(np.ceil(rec[P_MY] + r)) + 1, h))


def _union(a, b):
    if a is None:
        return b
    if b is None:
        return a
    return (min(a[0], b[0]), min(a[1], b[1]), max(a[2], b[2]), max(a[3], b[3]))


def _reorder(order_all: np.ndarray, keys: np.ndarray, i: int, new_key: float, valid: bool):
    """Compositing order with Gaussian i moved to its new depth key (or removed)."""
    o = order_all[order_all != i]
    if not valid:
        return o
    k = np.float32(new_key)
    ko = keys[o]
    # first position whose (key, index) is greater than (k, i)
    pos = np.searchsorted(ko, k, side="left")
    while pos < o.shape[0] and ko[pos] == k and o[pos] < i:
        pos += 1
    return np.insert(o, pos, i)


def fd_grad(g: dict, cam: dict, target_u8: np.ndarray, items, rel_h: float = 1e-5, proj=None,
            loss_mask=None):
    """Central finite differences of the L1 loss for (index, name, component) items.

    The loss change caused by one Gaussian is confined to its footprint, so
    only the pixels of the union of the footprints at theta, theta +- h are
    re-composited, with the compositing order of the other Gaussians kept, and
    the loss difference is summed per pixel (unchanged pixels cancel exactly).
    loss_mask (H x W bool, optional) restricts the loss sum to those pixels
    (same normalisation 1 / (3 H W)); only the footprint pixels inside the
    mask's bounding box are then re-composited.
    Returns (fd(h), fd(h/2)) arrays; entries where the two disagree sit on a
    kink (L1 sign flip, alpha clamp or gate, depth swap).
    """
    w, h = int(cam["width"]), int(cam["height"])
    base = {k: (np.array(v, dtype=np.float64, copy=True) if isinstance(v, np.ndarray) else v)
            for k, v in g.items()}
    # a private copy whose row i is swapped in place for each perturbed record
    proj = project(base, cam) if proj is None else np.array(proj, copy=True)
    order_all = order(proj)
    keys = proj[:, P_ZKEY].astype(np.float32)
    t = target_u8.astype(np.float64) / 255.0
    npix3 = w * h * 3
    box = None
    if loss_mask is not None:
        ys, xs = np.nonzero(loss_mask)
        box = (int(xs.min()), int(ys.min()), int(xs.max()) + 1, int(ys.max()) + 1) if ys.size else (0, 0, 0, 0)
    res = []
    for step_scale in (1.0, 0.5):
        vals = []
        for (i, name, comp) in items:
            arr = base[name]
            flat_idx = np.unravel_index(comp, arr.shape[1:]) if arr.ndim > 1 else ()
            theta = float(arr[(i,) + tuple(flat_idx)])
            hh = rel_h * max(1.0, abs(theta)) * step_scale
            one = {k: (v[i:i + 1].copy() if isinstance(v, np.ndarray) else v) for k, v in base.items()}
            recs = []
            for sgn in (+1, -1):
                one[name][(0,) + tuple(flat_idx)] = theta + sgn * hh
                recs.append(project(one, cam)[0])
            region = _union(_union(_footprint(proj[i], w, h), _footprint(recs[0], w, h)),
                            _footprint(recs[1], w, h))
            if region is not None and box is not None:
                region = (max(region[0], box[0]), max(region[1], box[1]), min(region[2], box[2]),
                          min(region[3], box[3]))
            if region is None or region[0] >= region[2] or region[1] >= region[3]:
                vals.append(0.0)
                continue
            losses = []
            saved, saved_key = proj[i].copy(), keys[i]
            x0, y0, x1, y1 = region
            for rec in recs:
                proj[i] = rec
                keys[i] = np.float32(rec[P_ZKEY])
                o = _reorder(order_all, keys, i, rec[P_ZKEY], rec[P_VALID] != 0)
                out = render(base, cam, region=region, proj=proj, order=o)
                losses.append(out["rgb"][y0:y1, x0:x1])
            proj[i], keys[i] = saved, saved_key
            # difference per pixel first: pixels the step leaves alone give exact zeros
            tt = t[y0:y1, x0:x1]
            dpix = np.abs(losses[0] - tt) - np.abs(losses[1] - tt)
            if loss_mask is not None:
                dpix = dpix * loss_mask[y0:y1, x0:x1, None]
            dl = dpix.sum()
            vals.append(dl / (2.0 * hh) / npix3)
        res.append(np.array(vals))
    return res[0], res[1]
