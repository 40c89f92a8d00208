"""Adam as a per-position gain controller (Algorithm 1 and Eqs. 8-9).

The measured registration shift g_j takes the place of the gradient in
Kingma & Ba's Algorithm 1; the moments are kept per position and per axis,
and the position moves by the bias-corrected step (a gain that adapts per
position).  Sign: g_j is the shift that moves position j toward where the data
put it, so the step is ADDED (pos += step), see ``rpie.iterate``.
"""
import numpy as np


def adam_step(pos, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8, max_step=0.0):
    """One Adam step for every position; t is the 1-based step count.

    Returns (new_pos, new_m, new_v), all float64 (N, 2).
    """
    g = np.asarray(g, dtype=np.float64)
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    step = lr * mhat / (np.sqrt(vhat) + eps)
    if max_step > 0:
        step = np.clip(step, -max_step, max_step)
    return pos + step, m, v
