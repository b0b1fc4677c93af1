"""FP64 reference of the learned reconstruction selector (TEST INFRASTRUCTURE).

The selector is not in the paper: it is a 15 -> 32 -> 32 -> 1 perceptron with
GELU activations (tanh form, 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))))
that reads the normalised five-point characteristic stencils of a face and
predicts whether WENO5-JS is needed (logit high) or the linear 5th-order
reconstruction suffices.  Training minimises the binary cross-entropy with
logits, weighted by `pos_weight` on the "WENO needed" class, averaged over the
batch; the optimiser is Adam (Kingma & Ba 2015).

BF16 operands: the GPU rounds inputs, weights and hidden activations to
bfloat16 and accumulates in FP32.  This reference applies the same roundings
(round to nearest even on the upper 16 bits) and accumulates in FP64, so that
GPU and reference differ only by the accumulation precision.  Pinned by
central finite differences on the unrounded network, and against torch's own
Linear / GELU(tanh) / BCEWithLogitsLoss layers with autograd, its bfloat16
conversion and its Adam optimiser (tests/test_oracle_mlp.py).

Parameter vector layout (1601 floats): W1[32][15] (out x in), b1[32],
W2[32][32], b2[32], w3[32], b3[1].
"""
from __future__ import annotations

import numpy as np

NIN, NH = 15, 32
SIZES = [("W1", (NH, NIN)), ("b1", (NH,)), ("W2", (NH, NH)), ("b2", (NH,)), ("w3", (NH,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)
K0 = np.sqrt(2.0 / np.pi)
K1 = 0.044715


def unpack(theta):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def bf16(x):
    """Round to bfloat16 (nearest even), returned as float64."""
    x32 = np.asarray(x, dtype=np.float32)
    b = x32.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    t = np.tanh(K0 * (z + K1 * z ** 3))
    return 0.5 * z * (1.0 + t)


def gelu_grad(z):
    t = np.tanh(K0 * (z + K1 * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * K0 * (1.0 + 3.0 * K1 * z * z)


def forward(theta, X, rounded=True):
    """Logits [n] and the cached activations."""
    p = unpack(theta)
    r = bf16 if rounded else (lambda a: np.asarray(a, dtype=np.float64))
    W1, W2, w3 = r(p["W1"]), r(p["W2"]), r(p["w3"])
    x = r(X)
    z1 = x @ W1.T + p["b1"]
    h1 = r(gelu(z1))
    z2 = h1 @ W2.T + p["b2"]
    h2 = r(gelu(z2))
    z3 = h2 @ w3 + p["b3"][0]
    return z3, dict(x=x, z1=z1, h1=h1, z2=z2, h2=h2, W1=W1, W2=W2, w3=w3)


def loss_and_grad(theta, X, y, pos_weight=1.0, rounded=True):
    """Mean weighted BCE-with-logits and its gradient w.r.t. theta (the
    gradient of the rounded network with respect to the rounded weights,
    i.e. the straight-through convention of mixed-precision training)."""
    n = X.shape[0]
    z, c = forward(theta, X, rounded)
    y = np.asarray(y, dtype=np.float64)
    w = np.where(y > 0.5, pos_weight, 1.0)
    L = w * (np.maximum(z, 0.0) - z * y + np.log1p(np.exp(-np.abs(z))))
    loss = L.mean()
    sig = 1.0 / (1.0 + np.exp(-z))
    dz3 = w * (sig - y) / n
    g = {}
    g["w3"] = c["h2"].T @ dz3
    g["b3"] = np.array([dz3.sum()])
    dh2 = np.outer(dz3, c["w3"])
    dz2 = dh2 * gelu_grad(c["z2"])
    g["W2"] = dz2.T @ c["h1"]
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ c["W2"]
    dz1 = dh1 * gelu_grad(c["z1"])
    g["W1"] = dz1.T @ c["x"]
    g["b1"] = dz1.sum(axis=0)
    return loss, pack(g)


def adam(theta, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns the new (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def init(seed=0):
    """Seeded initialisation: N(0, 1/fan_in) weights, zero biases."""
    rng = np.random.Generator(np.random.Philox(key=seed))
    d = {"W1": rng.normal(0, 1 / np.sqrt(NIN), (NH, NIN)), "b1": np.zeros(NH),
         "W2": rng.normal(0, 1 / np.sqrt(NH), (NH, NH)), "b2": np.zeros(NH),
         "w3": rng.normal(0, 1 / np.sqrt(NH), NH), "b3": np.zeros(1)}
    return pack(d)
