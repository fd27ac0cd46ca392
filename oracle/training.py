"""Oracle for the D2NN training step of Sec. 2.5 (TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``).

Plain numpy, FP64, written independently of the package: Adam (Kingma & Ba 2015) as published, the
one-cycle learning-rate schedule with cosine annealing (Smith & Topin 2019; the paper names the
schedule and lr = 0.01), and one epoch (propagation through the oracle's screens, the two-mask
receiver, MAE loss against the reference intensity, receiver adjoint, one Adam step per mask).
Pinned by ``tests/test_oracle_training.py`` (constant-gradient Adam steps of lr * sign(g), the
schedule's start / peak / end values).
"""
from __future__ import annotations

import math

import numpy as np


def adam(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t >= 1); returns the new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mhat = m / (1 - b1 ** t)
    vhat = v / (1 - b2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def one_cycle(step, total, lr_max, pct_start=0.3, div_factor=25.0, final_div_factor=1e4):
    """Cosine one-cycle: lr_max/div_factor -> lr_max at step pct_start*total - 1 -> that / final_div_factor
    at step total - 1."""
    start = lr_max / div_factor
    end = start / final_div_factor
    peak_at = pct_start * total - 1.0
    if step <= peak_at:
        x = step / peak_at
        return lr_max + (start - lr_max) * (1 + math.cos(math.pi * x)) / 2
    x = (step - peak_at) / (total - 1 - peak_at)
    return end + (lr_max - end) * (1 + math.cos(math.pi * x)) / 2


def epoch(O, md, dz, cn2, seed, e, source, A, th1, th2, Iref, state, t, lr, kind=0, scale=1.0):
    """One training epoch on realization e with the oracle's own building blocks (O = the oracle
    module; kind 0 = MAE, 1 = squared error; the loss and its gradient times `scale`): returns
    (loss, th1, th2, state)."""
    phis = np.stack([O.make_screen(md, cn2[s], dz[s], 0, seed, s, e) for s in range(len(dz))])
    U = O.propagate(md, dz, phis, source)
    I, Z1, W2, V = O.d2nn_forward(A, th1, th2, U)
    loss, dLdI = O.intensity_loss(I, Iref, kind, I.size)
    loss, dLdI = loss * scale, dLdI * scale
    g1, g2 = np.zeros_like(th1), np.zeros_like(th2)
    O.d2nn_backward(A, th1, th2, Z1, W2, V, dLdI, g1, g2)
    (m1, v1, m2, v2) = state
    th1, m1, v1 = adam(th1, g1, m1, v1, t, lr)
    th2, m2, v2 = adam(th2, g2, m2, v2, t, lr)
    return loss, th1, th2, (m1, v1, m2, v2)
