"""Seeded synthetic inputs for the edge-guided densification path.

This module is shared by the FP64 oracle tests, the CUDA parity tests and the
benchmark.  It holds random draws and camera placement only; none of the
method's arithmetic (edge map, splatting, split) lives here.

The paper evaluates on Mip-NeRF360 (Sec. 3.1), which is not available; these
generators stand in for it with scenes of the same shapes:

* images: a linear gradient between two random colours, 8 axis-aligned
  rectangles and 8 discs of uniform random colour, plus N(0, 2/255) noise,
  rounded to uint8, HWC layout;
* Gaussians: means U[-1,1]^3, log-scales N(-3, 0.5), quaternions normalised
  N(0, I4) stored (w, x, y, z), opacity logits N(0, 1), SH colour whose base
  colour c0 is U[0,1] (stored as DC = (c0 - 0.5) / Y00) and whose higher
  coefficients are N(0, 0.2);
* cameras: pinhole with a 60 degree field of view across the longer side,
  principal point at the image centre; a frontal camera at (0, 0, -4) looking
  along +z, or a ring of radius 4 around the origin with world up = -y.

Seeds follow one numpy PCG64 stream per object: image seed 1000 + view,
target seed 2000 + view, Gaussians seed 1.
"""
from __future__ import annotations

import math

import numpy as np

Y00 = 0.28209479177387814  # 1 / (2 sqrt(pi)); only used to store the base colour

RING_RESOLUTIONS = [(640, 480), (800, 600), (1024, 768), (1237, 822),
                    (1237, 822), (1440, 960), (1600, 1060), (1920, 1080)]


def image(height: int, width: int, seed: int) -> np.ndarray:
    """uint8 [H, W, 3] synthetic photograph (gradient + rectangles + discs + noise)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c0 = rng.uniform(0.0, 1.0, 3)
    c1 = rng.uniform(0.0, 1.0, 3)
    ys = np.arange(height, dtype=np.float64)[:, None]
    xs = np.arange(width, dtype=np.float64)[None, :]
    t = 0.5 * (xs / max(width - 1, 1) + ys / max(height - 1, 1))
    img = c0[None, None, :] * (1.0 - t[..., None]) + c1[None, None, :] * t[..., None]
    for _ in range(8):
        xa, xb = np.sort(rng.integers(0, width, 2))
        ya, yb = np.sort(rng.integers(0, height, 2))
        img[ya:yb + 1, xa:xb + 1, :] = rng.uniform(0.0, 1.0, 3)
    for _ in range(8):
        cx = rng.uniform(0, width)
        cy = rng.uniform(0, height)
        r = rng.uniform(0.03, 0.15) * min(width, height)
        col = rng.uniform(0.0, 1.0, 3)
        inside = (xs + 0.5 - cx) ** 2 + (ys + 0.5 - cy) ** 2 <= r * r
        img[inside] = col
    img = img + rng.normal(0.0, 2.0 / 255.0, img.shape)
    return np.clip(np.rint(img * 255.0), 0, 255).astype(np.uint8)


def gaussians(n: int, sh_degree: int, seed: int = 1) -> dict:
    """Float32 SoA parameter set of n Gaussians (caller-owned storage layout)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    k = (sh_degree + 1) ** 2
    means = rng.uniform(-1.0, 1.0, (n, 3))
    log_scales = rng.normal(-3.0, 0.5, (n, 3))
    q = rng.normal(0.0, 1.0, (n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opacity_logits = rng.normal(0.0, 1.0, n)
    sh = np.zeros((n, k, 3))
    sh[:, 0, :] = (rng.uniform(0.0, 1.0, (n, 3)) - 0.5) / Y00
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.2, (n, k - 1, 3))
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return {"means": f32(means), "log_scales": f32(log_scales), "quats": f32(q),
            "opacity_logits": f32(opacity_logits), "sh": f32(sh), "sh_degree": sh_degree}


def _focal(width: int, height: int) -> float:
    return (max(width, height) / 2.0) / math.tan(math.radians(30.0))


def camera_look_at(center, width: int, height: int) -> dict:
    """Camera at `center` looking at the origin, world up = -y (image y points down)."""
    c = np.asarray(center, dtype=np.float64)
    f = -c / np.linalg.norm(c)
    down = np.array([0.0, 1.0, 0.0])
    x = np.cross(down, f)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    rot = np.stack([x, y, f])
    t = -rot @ c
    viewmat = np.concatenate([rot, t[:, None]], axis=1).astype(np.float32)
    fl = _focal(width, height)
    return {"viewmat": viewmat, "fx": np.float32(fl), "fy": np.float32(fl),
            "cx": np.float32(width / 2.0), "cy": np.float32(height / 2.0),
            "width": int(width), "height": int(height)}


def camera_front(width: int, height: int) -> dict:
    """Camera at (0, 0, -4), identity rotation, looking along +z."""
    return camera_look_at((0.0, 0.0, -4.0), width, height)


def camera_ring(k: int, n: int = 8, radius: float = 4.0, resolutions=None) -> dict:
    """Camera k of n on a ring of the given radius in the xz-plane."""
    res = resolutions or RING_RESOLUTIONS
    w, h = res[k % len(res)]
    th = 2.0 * math.pi * k / n
    return camera_look_at((radius * math.cos(th), 0.0, radius * math.sin(th)), w, h)
