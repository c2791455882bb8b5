"""FP64 oracle of the optimiser step and the learning-rate schedule.

TEST INFRASTRUCTURE ONLY (tests/, the smoke test, the benchmark's CPU leg).

The paper does not state its optimiser; the densification loop uses plain
SGD.  Its learning-rate schedule (Sec. 2.3, "Refinement Setup" and
"Positional Learning Rate Optimization") is an exponential decay per
parameter group from an initial to a final rate: the scale rate from 0.020 to
0.002 (gamma = 0.1), the positional rate from 1.28e-4 to 1.28e-5.  Reading:
lr(t) = lr_init * (lr_final / lr_init) ** (min(t, steps) / steps), the rate
constant after `steps` (the paper does not state the horizon).
"""
from __future__ import annotations

import numpy as np

GROUPS = ("means", "log_scales", "quats", "opacity_logits", "sh")
PAPER_SCHEDULE = {"means": (1.28e-4, 1.28e-5), "log_scales": (0.020, 0.002)}


def lr_at(lr_init: float, lr_final: float, steps: int, t: int) -> float:
    """Rate of one group at step t (exponential interpolation, held after steps)."""
    if lr_init == lr_final:
        return float(lr_init)
    frac = min(max(int(t), 0), int(steps)) / float(steps)
    return float(lr_init) * (float(lr_final) / float(lr_init)) ** frac


def sgd_step(params: dict, grads: dict, lrs: dict, n: int) -> dict:
    """theta - lr * grad on rows [0, n) of every group (FP64)."""
    out = {k: np.array(v, dtype=np.float64) for k, v in params.items()}
    for k in GROUPS:
        out[k][:n] = out[k][:n] - lrs[k] * np.asarray(grads[k], dtype=np.float64)[:n]
    return out
