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

Gradient-threshold candidate masking (Sec. 2.3, "Global Warm-up Phase"; the
paper names the masking but not its statistic nor its threshold).  Reading:
the positional statistic of Gaussian i is the mean, over the (iteration,
view) pairs in which its screen-space mean gradient is nonzero, of that
gradient's Euclidean norm; i is a candidate when it has at least one such
pair and the mean is >= tau.  The selection then takes the top-k edge scores
among the candidates (fewer when there are fewer candidates).  The first
three densification events skip the masking (the warm-up).  The candidate
decision is an integer one taken from floating point: it is taken in FP32,
mean = float32(sum) / float32(count), the precision of the kernel.
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


def pos_grad_stats(g2d_views, sums=None, counts=None):
    """Accumulate the positional statistic over views: g2d_views is a list of
    (n, >= 2) arrays of screen-space gradients whose columns 0, 1 are
    dL/d(mean2D x, y).  Returns (sum of norms, number of nonzero views)."""
    g0 = np.asarray(g2d_views[0])
    n = g0.shape[0]
    s = np.zeros(n) if sums is None else np.array(sums, dtype=np.float64)
    c = np.zeros(n, dtype=np.int64) if counts is None else np.array(counts, dtype=np.int64)
    for g in g2d_views:
        g = np.asarray(g, dtype=np.float64)
        nz = (g[:, 0] != 0) | (g[:, 1] != 0)
        s[nz] += np.hypot(g[nz, 0], g[nz, 1])
        c[nz] += 1
    return s, c


def grad_candidates(sums: np.ndarray, counts: np.ndarray, tau: float) -> np.ndarray:
    """Candidates of the gradient-threshold masking (decision in FP32)."""
    sums32 = np.asarray(sums, dtype=np.float32)
    c = np.asarray(counts, dtype=np.int64)
    with np.errstate(divide="ignore", invalid="ignore"):
        mean = sums32 / np.maximum(c, 1).astype(np.float32)
    return (c > 0) & (mean >= np.float32(tau))


def gated_topk_mask(scores: np.ndarray, k: int, sums: np.ndarray, counts: np.ndarray, tau: float) -> np.ndarray:
    """Top-k by score among the gradient-threshold candidates (ties toward the
    lower index); selects min(k, number of candidates)."""
    cand = grad_candidates(sums, counts, tau)
    idx = np.nonzero(cand)[0]
    sub = topk_mask(np.asarray(scores)[idx], k)
    mask = np.zeros(np.asarray(scores).shape[0], dtype=bool)
    mask[idx[sub]] = True
    return mask


def sample_mask(scores: np.ndarray, expv: np.ndarray, k: int) -> np.ndarray:
    """Importance sampling by edge score (Sec. 1, "Edge-Score importance
    sampling"): k Gaussians drawn without replacement with probabilities
    proportional to their scores, by exponential clocks: Gaussian i rings at
    expv[i] / scores[i] (expv: independent Exp(1) variates, an input), the k
    earliest are taken (ties toward the lower index); scores <= 0 never ring.
    The ringing times are FP32 quotients, the precision of the kernel."""
    s = np.asarray(scores, dtype=np.float32)
    e = np.asarray(expv, dtype=np.float32)
    live = np.nonzero(s > 0)[0]
    t = e[live] / s[live]  # float32 / float32: one IEEE division
    sub = topk_mask(-t, k)
    mask = np.zeros(s.shape[0], dtype=bool)
    mask[live[sub]] = True
    return mask


def budgeted_k(k: int, n: int, budget: int) -> int:
    """Selections allowed under a Gaussian budget (Conclusion: 1M-budget variant):
    the split adds one Gaussian per selection, so at most budget - n (budget 0:
    no budget)."""
    return int(k) if budget <= 0 else max(0, min(int(k), int(budget) - int(n)))


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
