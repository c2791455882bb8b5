"""FP64 oracle of the edge-importance map (paper Sec. 2.1).

TEST INFRASTRUCTURE ONLY: this module is imported by tests/, by the smoke test
of __graft_entry__ and by the CPU-baseline leg of bench.py.  The product path
never calls it.

The paper lists the stages (Sec. 2.1, steps 1-3 and the closing paragraph):
grayscale conversion and a 5x5 Gaussian blur, Sobel magnitude and orientation,
non-maximum suppression along the gradient, then division by the median.  It
leaves the numeric details open; the readings used here are:

* luma weights 0.299 / 0.587 / 0.114 applied to the uint8 values, divided by 255;
* border: the grayscale image is extended beyond its edges by clamp-to-edge
  (edge replication); the blur and the Sobel filters then act on that
  extended image, so no second clamp happens between them;
* blur taps w_k = exp(-k^2 / (2 sigma^2)), k = -2..2, normalised to sum 1, the
  2-D kernel being w (x) w;
* Sobel gx = [[-1,0,1],[-2,0,2],[-1,0,1]] correlated with the blurred image,
  gy its transpose (image y points down), M = |(gx, gy)|_2;
* NMS: the gradient vector is quantised to 8 directions.  With ax = |gx|,
  ay = |gy| and t = tan(22.5 deg) = sqrt(2) - 1: horizontal if ay <= t*ax,
  vertical if ax <= t*ay, diagonal otherwise.  n+ is the neighbour one step
  uphill along that direction (signs of gx, gy), n- the opposite one; pixels
  outside the image count as magnitude 0.  A pixel is kept iff
  M > 0 and M >= M(n+) and M > M(n-);
* median: the lower median (element floor((n-1)/2) of the ascending sort) of
  the kept magnitudes; E = M_thinned / median, and E = 0, median = 0 when no
  pixel is kept.

Every function works on one view; the batched kernels apply it per view.
"""
from __future__ import annotations

import math

import numpy as np

LUMA = (0.299, 0.587, 0.114)
TAN22 = math.sqrt(2.0) - 1.0


def gray(rgb_u8: np.ndarray) -> np.ndarray:
    """Sec. 2.1 step 1: luma of an HWC uint8 image, scaled to [0, 1]."""
    x = rgb_u8.astype(np.float64)
    return (LUMA[0] * x[..., 0] + LUMA[1] * x[..., 1] + LUMA[2] * x[..., 2]) / 255.0


def blur_taps(sigma: float = 1.0) -> np.ndarray:
    """Sec. 2.1 step 1: 1-D taps of the 5x5 Gaussian (normalised to sum 1)."""
    k = np.arange(-2, 3, dtype=np.float64)
    w = np.exp(-(k * k) / (2.0 * sigma * sigma))
    return w / w.sum()


def extend(y: np.ndarray, pad: int = 3) -> np.ndarray:
    """Grayscale image extended by `pad` pixels of clamp-to-edge replication."""
    return np.pad(y, pad, mode="edge")


def _window(img: np.ndarray, dy: int, dx: int, crop: int) -> np.ndarray:
    """img[y+dy, x+dx] over the interior that is `crop` pixels inside img."""
    h, w = img.shape
    return img[crop + dy:h - crop + dy, crop + dx:w - crop + dx]


def blur(y_ext: np.ndarray, taps: np.ndarray) -> np.ndarray:
    """Sec. 2.1 step 1: 2-D correlation with taps (x) taps.

    Takes the image extended by 3 pixels and returns it extended by 1 pixel
    (the Sobel stage needs one ring of blurred values around the image).
    """
    out = np.zeros((y_ext.shape[0] - 4, y_ext.shape[1] - 4))
    for a in range(-2, 3):
        for b in range(-2, 3):
            out += taps[a + 2] * taps[b + 2] * _window(y_ext, a, b, 2)
    return out


SOBEL_X = np.array([[-1.0, 0.0, 1.0], [-2.0, 0.0, 2.0], [-1.0, 0.0, 1.0]])
SMOOTH = (1.0, 2.0, 1.0)


def sobel(b_ext: np.ndarray):
    """Sec. 2.1 step 2: (gx, gy, M) from the blurred image extended by 1 pixel.

    gx is the correlation with SOBEL_X, written as the [1, 2, 1]-weighted sum
    of central differences b(x+1) - b(x-1) (the same operator; flat regions
    give exactly 0); gy is the transposed operator.
    """
    shape = (b_ext.shape[0] - 2, b_ext.shape[1] - 2)
    gx = np.zeros(shape)
    gy = np.zeros(shape)
    for k in range(-1, 2):
        gx += SMOOTH[k + 1] * (_window(b_ext, k, 1, 1) - _window(b_ext, k, -1, 1))
        gy += SMOOTH[k + 1] * (_window(b_ext, 1, k, 1) - _window(b_ext, -1, k, 1))
    return gx, gy, np.sqrt(gx * gx + gy * gy)


def direction_step(gx: np.ndarray, gy: np.ndarray):
    """Quantised uphill step (sx, sy) in {-1,0,1}^2 for each pixel (Sec. 2.1 step 3)."""
    ax, ay = np.abs(gx), np.abs(gy)
    horiz = ay <= TAN22 * ax
    vert = (~horiz) & (ax <= TAN22 * ay)
    sx = np.where(vert, 0, np.sign(gx)).astype(np.int64)
    sy = np.where(horiz, 0, np.sign(gy)).astype(np.int64)
    return sx, sy


def nms(m: np.ndarray, gx: np.ndarray, gy: np.ndarray):
    """Sec. 2.1 step 3: thinned magnitude and keep-mask.

    Returns (m_thin, keep, m_plus, m_minus); m_plus / m_minus are the compared
    neighbour magnitudes (0 outside the image), used by the tolerance rule.
    """
    h, w = m.shape
    sx, sy = direction_step(gx, gy)
    yy, xx = np.mgrid[0:h, 0:w]

    def sample(ox, oy):
        x2, y2 = xx + ox, yy + oy
        ok = (x2 >= 0) & (x2 < w) & (y2 >= 0) & (y2 < h)
        return np.where(ok, m[np.clip(y2, 0, h - 1), np.clip(x2, 0, w - 1)], 0.0)

    m_plus = sample(sx, sy)
    m_minus = sample(-sx, -sy)
    keep = (m > 0.0) & (m >= m_plus) & (m > m_minus)
    return np.where(keep, m, 0.0), keep, m_plus, m_minus


def lower_median(values: np.ndarray) -> float:
    """Element floor((n-1)/2) of the ascending sort; 0 for an empty set."""
    v = np.sort(values.ravel())
    return float(v[(v.size - 1) // 2]) if v.size else 0.0


def edge_map_gray(y: np.ndarray, taps: np.ndarray | None = None) -> dict:
    """Edge-importance map of one grayscale view (Sec. 2.1 steps 1-3 + median)."""
    taps = blur_taps(1.0) if taps is None else np.asarray(taps, dtype=np.float64)
    b = blur(extend(y, 3), taps)
    gx, gy, m = sobel(b)
    m_thin, keep, m_plus, m_minus = nms(m, gx, gy)
    med = lower_median(m_thin[keep])
    e = m_thin / med if med > 0.0 else np.zeros_like(m_thin)
    return {"E": e, "median": med, "keep": keep, "M": m, "gx": gx, "gy": gy,
            "blur": b[1:-1, 1:-1], "m_plus": m_plus, "m_minus": m_minus}


def edge_map(rgb_u8: np.ndarray, taps: np.ndarray | None = None) -> dict:
    """Edge-importance map of one HWC uint8 view."""
    return edge_map_gray(gray(rgb_u8), taps)


def nms_exempt(out: dict, rel: float = 1e-6) -> np.ndarray:
    """Pixels whose keep decision rests on a near-tie.

    A pixel is exempt when one of its compared magnitude pairs (M vs M(n+),
    M vs M(n-)) or its direction-bin boundary test (|gy| vs t|gx|, |gx| vs
    t|gy|) differs by less than `rel` relative; FP32 and FP64 may take such a
    decision differently.
    """
    m, mp, mm = out["M"], out["m_plus"], out["m_minus"]
    ax, ay = np.abs(out["gx"]), np.abs(out["gy"])

    def close(a, b):
        return np.abs(a - b) <= rel * np.maximum(np.abs(a), np.abs(b))

    ex = (close(m, mp) & (m > 0)) | (close(m, mm) & (m > 0))
    ex |= (close(ay, TAN22 * ax) | close(ax, TAN22 * ay)) & (m > 0)
    ex |= (m > 0) & (m <= rel * np.max(m, initial=0.0))
    return ex
