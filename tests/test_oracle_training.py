"""Training-loop oracle (Sec. 2.5) against closed forms, and the package's one-cycle schedule against
it (CPU only)."""
import math

import numpy as np
import pytest

from oracle import training as T


def test_adam_with_a_constant_gradient_moves_lr_per_step():
    # m_hat = g and v_hat = g^2 exactly for a constant g, so each step moves p by lr g / (|g| + eps)
    g = np.array([2.0, -0.5, 1e-3])
    p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for t in range(1, 6):
        p, m, v = T.adam(p, g, m, v, t, lr=0.01)
        assert np.allclose(p, -0.01 * t * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_adam_first_step_is_lr_times_sign():
    rng = np.random.default_rng(0)
    g = rng.standard_normal(100)
    p, _, _ = T.adam(np.zeros(100), g, np.zeros(100), np.zeros(100), 1, lr=0.05)
    assert np.allclose(p, -0.05 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_one_cycle_start_peak_end():
    total, lr = 20000, 0.01
    assert T.one_cycle(0, total, lr) == pytest.approx(lr / 25, rel=1e-12)
    assert T.one_cycle(0.3 * total - 1, total, lr) == pytest.approx(lr, rel=1e-12)
    assert T.one_cycle(total - 1, total, lr) == pytest.approx(lr / 25 / 1e4, rel=1e-12)
    # halfway up and halfway down are the arithmetic means of the phase's ends (cosine)
    assert T.one_cycle((0.3 * total - 1) / 2, total, lr) == pytest.approx((lr + lr / 25) / 2, rel=1e-12)
    mid_down = (0.3 * total - 1 + total - 1) / 2
    assert T.one_cycle(mid_down, total, lr) == pytest.approx((lr + lr / 25e4) / 2, rel=1e-12)
    lrs = [T.one_cycle(s, total, lr) for s in range(total)]
    peak = int(np.argmax(lrs))
    assert abs(peak - (0.3 * total - 1)) <= 1
    assert all(a <= b for a, b in zip(lrs[:peak], lrs[1:peak + 1]))
    assert all(a >= b for a, b in zip(lrs[peak:-1], lrs[peak + 1:]))


def test_package_schedule_matches_oracle():
    tr = pytest.importorskip("paper_2604_07248_gb300.training")
    for total in (10, 777, 20000):
        for s in range(0, total, max(1, total // 97)):
            assert math.isclose(tr.one_cycle_lr(s, total, 0.01), T.one_cycle(s, total, 0.01), rel_tol=1e-12)
