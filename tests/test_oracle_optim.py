"""Pins of the oracle's Adam step against closed forms."""
import numpy as np

from oracle import optim


def test_first_step_moves_by_lr_times_sign():
    # t = 1 from zero moments: m_hat = g, v_hat = g^2, step = lr g / (|g| + eps)
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    p, m, v = optim.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.1, eps=0.0 + 1e-12)
    np.testing.assert_allclose(p[:3], -0.1 * np.sign(g[:3]), rtol=1e-8)
    assert p[3] == 0.0
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_constant_gradient_keeps_unit_steps():
    # with a constant gradient the bias-corrected ratio stays g/|g| at every step
    p = np.zeros(1)
    m = np.zeros(1)
    v = np.zeros(1)
    for t in range(1, 20):
        p_prev = p.copy()
        p, m, v = optim.adam_step(p, np.array([2.0]), m, v, t, lr=0.01, eps=1e-12)
        np.testing.assert_allclose(p_prev - p, [0.01], rtol=1e-9)


def test_clamps():
    p, _, _ = optim.adam_step(np.array([0.02, 1.99]), np.array([1.0, -1.0]), np.zeros(2), np.zeros(2), 1,
                              lr=0.5, lo=0.01, hi=2.0)
    np.testing.assert_array_equal(p, [0.01, 2.0])


def test_grid_step_schedule_end_points_and_midpoint():
    # Eq. 14: h_max before t_b, h_min after t_e, the mean at the middle, monotone
    from oracle.optim import grid_step
    args = dict(T=300, h_max=4.0, h_min=1.0, t_b=0.1, t_e=0.8)
    assert grid_step(0, **args) == 4.0 and grid_step(30, **args) == 4.0
    assert grid_step(240, **args) == 1.0 and grid_step(299, **args) == 1.0
    assert abs(grid_step(135, **args) - 2.5) < 1e-12          # phi = 1/2
    hs = [grid_step(t, **args) for t in range(300)]
    assert all(a >= b for a, b in zip(hs, hs[1:]))
