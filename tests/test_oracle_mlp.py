"""Pins of the selector's FP64 reference (oracle/mlp.py): central finite
differences of the loss, the BF16 rounding rule, and one Adam step by hand."""
import numpy as np

from oracle import mlp


def test_gradient_central_differences():
    rng = np.random.default_rng(0)
    theta = mlp.init(3) + rng.normal(0, 0.05, mlp.NPARAM)
    X = rng.uniform(-1, 1, (40, 15))
    y = (rng.uniform(size=40) < 0.3).astype(float)
    loss, g = mlp.loss_and_grad(theta, X, y, pos_weight=4.0, rounded=False)
    h = 1e-6
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    for i in list(idx) + [mlp.NPARAM - 1, 0, 480, 512]:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, X, y, 4.0, rounded=False)[0] - mlp.loss_and_grad(tm, X, y, 4.0, rounded=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_bf16_rounding():
    # representable values are unchanged; halfway cases round to even
    x = np.array([1.0, -2.5, 0.0, 1.0 + 2 ** -7, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8])
    r = mlp.bf16(x)
    assert r[0] == 1.0 and r[1] == -2.5 and r[2] == 0.0 and r[3] == 1.0 + 2 ** -7
    assert r[4] == 1.0                    # tie -> even mantissa
    assert r[5] == 1.0 + 2 ** -6          # tie -> even mantissa (up)


def test_adam_first_step_moves_by_lr():
    theta = np.zeros(4)
    g = np.array([1.0, -2.0, 0.5, 0.0])
    t2, m, v = mlp.adam(theta, g, np.zeros(4), np.zeros(4), 1, lr=0.1)
    # first step: m_hat = g, v_hat = g^2 -> update = lr * sign(g) (up to eps)
    assert np.allclose(t2[:3], -0.1 * np.sign(g[:3]), atol=1e-7)
    assert t2[3] == 0.0
