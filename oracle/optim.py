"""FP64 oracle, part 5: the Adam step with the parameter clamps of Table S1.

Test infrastructure only.  Adam (Kingma and Ba) written from its definition:
    m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2,
    p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),
followed by clamping p to [lo, hi] (the paper clamps weights to [0.01, 10]
and knot intervals to [0, 2]).
"""
import numpy as np


def adam_step(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8, lo=-np.inf, hi=np.inf):
    p = np.asarray(p, np.float64)
    g = np.asarray(g, np.float64)
    m = b1 * np.asarray(m, np.float64) + (1 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    p = np.clip(p - lr * mh / (np.sqrt(vh) + eps), lo, hi)
    return p, m, v


def grid_step(t, T, h_max, h_min, t_b, t_e):
    """Cosine grid-step annealing (Eq. 14): h = h_max + (h_min - h_max)(1 + cos(pi (1 - phi)))/2
    with phi = (t/T - t_b)/(t_e - t_b) inside (t_b, t_e), clamped outside."""
    import math
    f = t / T
    if f <= t_b:
        return h_max
    if f >= t_e:
        return h_min
    phi = (f - t_b) / (t_e - t_b)
    return h_max + (h_min - h_max) * (1 + math.cos(math.pi * (1 - phi))) / 2
