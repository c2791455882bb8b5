"""FP64 oracle of edge-score selection and Long-Axis-Split (paper Sec. 2.2).

TEST INFRASTRUCTURE ONLY (tests/, the smoke test, the benchmark's CPU leg).

Selection: the paper samples Gaussians by their edge score (Sec. 1); the
selection used here is the top-k by score: every Gaussian whose score is
above the k-th largest, plus the lowest-index ones among those equal to it.

Long-Axis-Split, Alg. 1 with the column read of Alg. 2, per selected Gaussian:
  l      = argmax of the (log) scale, first index on ties
  off    = k_off * exp(log_scale[l])          (physical scale, Alg. 1)
  scale  : log_scale[l] += log(long_factor); the others += log(other_factor)
  opac   : logit(beta * sigmoid(o))
  d      = R[:, l] * off, i.e. entries l, l+3, l+6 of the row-major R (Alg. 2)
  child 0 replaces the parent at mu + d; child 1 is appended at slot
  N + rank (rank = position among the selected, in index order) at mu - d;
  quaternion and SH are copied.
The paper's constants (Sec. 2.2, after Alg. 1) are k_off = alpha = 0.5,
long_factor = alpha = 0.5, other_factor = gamma = 0.85, beta = 0.6.
"""
from __future__ import annotations

import numpy as np

PAPER_PRESET = {"k_off": 0.5, "long_factor": 0.5, "other_factor": 0.85, "beta": 0.6}
CONFIG_PRESET = {"k_off": 1.0, "long_factor": 0.5, "other_factor": 1.0, "beta": 0.6}


def topk_mask(scores: np.ndarray, k: int) -> np.ndarray:
    """Top-k selection mask with ties broken toward the lower index."""
    s = np.asarray(scores)
    n = s.shape[0]
    k = max(0, min(int(k), n))
    order = np.lexsort((np.arange(n), -s.astype(np.float64)))
    mask = np.zeros(n, dtype=bool)
    mask[order[:k]] = True
    return mask


def quat_rot(q: np.ndarray) -> np.ndarray:
    q = q / np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def las_split(g: dict, mask: np.ndarray, k_off: float, long_factor: float, other_factor: float,
              beta: float) -> dict:
    """Apply Alg. 1 to the selected Gaussians; returns N + k parameter arrays (FP64)."""
    n = g["means"].shape[0]
    sel = np.nonzero(np.asarray(mask, dtype=bool))[0]
    out = {name: np.concatenate([np.asarray(g[name], dtype=np.float64),
                                 np.asarray(g[name], dtype=np.float64)[sel]], axis=0)
           for name in ("means", "log_scales", "quats", "opacity_logits", "sh")}
    out["sh_degree"] = g["sh_degree"]
    for rank, i in enumerate(sel):
        s = np.asarray(g["log_scales"][i], dtype=np.float64)
        l = int(np.argmax(s))
        off = k_off * np.exp(s[l])
        ns = s + np.log(other_factor)
        ns[l] = s[l] + np.log(long_factor)
        o = float(g["opacity_logits"][i])
        p = beta / (1.0 + np.exp(-o))
        no = np.log(p / (1.0 - p))
        rflat = quat_rot(np.asarray(g["quats"][i], dtype=np.float64)).ravel()
        d = np.array([rflat[l], rflat[l + 3], rflat[l + 6]]) * off
        mu = np.asarray(g["means"][i], dtype=np.float64)
        for slot, sign in ((i, 1.0), (n + rank, -1.0)):
            out["means"][slot] = mu + sign * d
            out["log_scales"][slot] = ns
            out["opacity_logits"][slot] = no
    return out
