"""Pins of the selector's FP64 reference (oracle/mlp.py): central finite
differences of the loss, the BF16 rounding rule, one Adam step by hand, and
the forward, loss, gradient, BF16 rounding and Adam steps against torch's own
layers, conversion and optimiser on the CPU."""
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


def _torch_net(theta):
    """The same 15-32-32-1 network written with torch's own layers (FP64, CPU)."""
    torch = __import__("pytest").importorskip("torch")
    p = mlp.unpack(theta)
    l1, l2, l3 = torch.nn.Linear(15, 32), torch.nn.Linear(32, 32), torch.nn.Linear(32, 1)
    with torch.no_grad():
        for lin, W, b in ((l1, p["W1"], p["b1"]), (l2, p["W2"], p["b2"]), (l3, p["w3"][None, :], p["b3"])):
            lin.weight = torch.nn.Parameter(torch.tensor(W, dtype=torch.float64))
            lin.bias = torch.nn.Parameter(torch.tensor(b, dtype=torch.float64))
    act = torch.nn.GELU(approximate="tanh")
    return torch, torch.nn.Sequential(l1, act, l2, act, l3)


def test_forward_loss_and_gradient_match_torch_layers():
    """Forward pass, weighted BCE-with-logits and backward pass of the
    unrounded network equal torch's Linear / GELU(tanh) / BCEWithLogitsLoss
    with autograd, which fixes the layer order, the parameter layout, the
    GELU form and the loss weighting independently of the finite differences."""
    rng = np.random.default_rng(3)
    theta = mlp.init(5) + rng.normal(0, 0.05, mlp.NPARAM)
    X = rng.uniform(-2, 2, (64, 15))
    y = (rng.uniform(size=64) < 0.3).astype(float)
    torch, net = _torch_net(theta)
    z_t = net(torch.tensor(X))[:, 0]
    z, _ = mlp.forward(theta, X, rounded=False)
    assert np.allclose(z, z_t.detach().numpy(), rtol=1e-13, atol=1e-13)
    lossf = torch.nn.BCEWithLogitsLoss(pos_weight=torch.tensor(4.0, dtype=torch.float64))
    L_t = lossf(z_t, torch.tensor(y))
    L_t.backward()
    loss, g = mlp.loss_and_grad(theta, X, y, pos_weight=4.0, rounded=False)
    assert abs(loss - L_t.item()) <= 1e-13 * abs(loss)
    l1, _, l2, _, l3 = net
    g_t = mlp.pack({"W1": l1.weight.grad.numpy(), "b1": l1.bias.grad.numpy(), "W2": l2.weight.grad.numpy(),
                    "b2": l2.bias.grad.numpy(), "w3": l3.weight.grad.numpy()[0], "b3": l3.bias.grad.numpy()})
    assert np.allclose(g, g_t, rtol=1e-10, atol=1e-14)


def test_bf16_rounding_matches_torch():
    """Round to nearest even on random and boundary values, against torch's
    own float -> bfloat16 conversion."""
    torch = __import__("pytest").importorskip("torch")
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.normal(0, 1, 20000) * 10.0 ** rng.uniform(-6, 6, 20000),
                        np.float32(1.0) + np.arange(-64, 64) * 2.0 ** -16])
    x32 = x.astype(np.float32)
    ref = torch.tensor(x32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x32), ref)


def test_adam_matches_torch_optimiser():
    """Five Adam steps with torch.optim.Adam's defaults apart from the rate."""
    torch = __import__("pytest").importorskip("torch")
    rng = np.random.default_rng(6)
    theta = rng.normal(0, 1, 10)
    grads = rng.normal(0, 1, (5, 10))
    p = torch.nn.Parameter(torch.tensor(theta))
    opt = torch.optim.Adam([p], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    m, v, th = np.zeros(10), np.zeros(10), theta.copy()
    for t in range(5):
        p.grad = torch.tensor(grads[t])
        opt.step()
        th, m, v = mlp.adam(th, grads[t], m, v, t + 1, lr=1e-2)
    assert np.allclose(th, p.detach().numpy(), rtol=1e-12, atol=1e-15)
