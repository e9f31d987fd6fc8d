"""Adam / AdamW update (Sec. 5.1 optimiser), FP64 (oracle; test infrastructure).

Standard Kingma-Ba moments with bias correction; decoupled weight decay (AdamW) applied as
p <- p - lr wd p before the moment step (the paper's decay value is not stated; the workloads use 0).
"""
from __future__ import annotations

import numpy as np


def adam_step(p, g, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
              weight_decay: float = 0.0):
    """One step at step count t >= 1; returns new (p, m, v) as float64 arrays."""
    p = np.asarray(p, np.float64)
    g = np.asarray(g, np.float64)
    p = p - lr * weight_decay * p
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
