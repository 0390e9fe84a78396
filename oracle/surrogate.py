"""FP64 CPU oracle of the surrogate network (TEST INFRASTRUCTURE ONLY).

A multilayer perceptron d_in -> H -> H -> H -> 1 with GELU activations,
gelu(z) = z Phi(z), the mean-squared loss and Adam (Kingma, Ba 2015), written
out with numpy in FP64.  With bf16=True the operands of the three hidden-layer
products -- exactly the ones the GPU feeds to its BF16 tensor cores -- are
rounded to BF16 first (round to nearest even), so that the GPU's forward pass and
gradient can be compared closely; with bf16=False it is the exact network.
The parameter vector has the GPU's order: W1, b1, W2, b2, W3, b3, w4, b4.
Pinned by central finite differences of the loss (tests/test_oracle_surrogate.py).
"""
import math

import numpy as np


def bf16_round(x):
    """Round to the nearest BF16 value (ties to even), returned as FP64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


_erf = np.vectorize(math.erf, otypes=[np.float64])


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    Phi = 0.5 * (1.0 + _erf(z / math.sqrt(2.0)))
    phi = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    return Phi + z * phi


def layout(d_in, H):
    sizes = [("W1", (H, d_in)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, H)),
             ("b3", (H,)), ("w4", (H,)), ("b4", (1,))]
    out, off = {}, 0
    for name, shape in sizes:
        n = int(np.prod(shape))
        out[name] = (off, shape)
        off += n
    return out, off


def unpack(p, d_in, H):
    lay, _ = layout(d_in, H)
    return {k: np.asarray(p[o:o + int(np.prod(s))], dtype=np.float64).reshape(s)
            for k, (o, s) in lay.items()}


def init_params(d_in, H, seed):
    """He-style initialisation (normal, variance 2 / fan_in), zero biases."""
    rng = np.random.default_rng(seed)
    lay, n = layout(d_in, H)
    p = np.zeros(n)
    for name, fan in (("W1", d_in), ("W2", H), ("W3", H), ("w4", H)):
        o, s = lay[name]
        p[o:o + int(np.prod(s))] = rng.normal(0.0, math.sqrt(2.0 / fan), size=int(np.prod(s)))
    return p


def _mm(a, b, bf16):
    if bf16:
        a, b = bf16_round(a), bf16_round(b)
    return a @ b


def forward(p, X, d_in, H, bf16=False):
    w = unpack(p, d_in, H)
    X = np.asarray(X, dtype=np.float64)
    Z1 = _mm(X, w["W1"].T, bf16) + w["b1"]
    A1 = gelu(Z1)
    Z2 = _mm(A1, w["W2"].T, bf16) + w["b2"]
    A2 = gelu(Z2)
    Z3 = _mm(A2, w["W3"].T, bf16) + w["b3"]
    A3 = gelu(Z3)
    y = A3 @ w["w4"] + w["b4"][0]
    return y, dict(X=X, Z1=Z1, A1=A1, Z2=Z2, A2=A2, Z3=Z3, A3=A3)


def loss_grad(p, X, t, d_in, H, bf16=False):
    """(loss, flat gradient) of mean (y - t)^2."""
    w = unpack(p, d_in, H)
    y, c = forward(p, X, d_in, H, bf16)
    B = len(t)
    e = y - np.asarray(t, dtype=np.float64)
    loss = float(np.mean(e * e))
    dy = 2.0 * e / B
    g = {}
    g["w4"] = c["A3"].T @ dy
    g["b4"] = np.array([dy.sum()])
    dZ3 = np.outer(dy, w["w4"]) * gelu_grad(c["Z3"])
    g["W3"] = _mm(dZ3.T, c["A2"], bf16)
    g["b3"] = dZ3.sum(0)
    dZ2 = _mm(dZ3, w["W3"], bf16) * gelu_grad(c["Z2"])
    g["W2"] = _mm(dZ2.T, c["A1"], bf16)
    g["b2"] = dZ2.sum(0)
    dZ1 = _mm(dZ2, w["W2"], bf16) * gelu_grad(c["Z1"])
    g["W1"] = _mm(dZ1.T, c["X"], bf16)
    g["b1"] = dZ1.sum(0)
    lay, n = layout(d_in, H)
    flat = np.zeros(n)
    for k, (o, s) in lay.items():
        flat[o:o + int(np.prod(s))] = g[k].ravel()
    return loss, flat


def adam(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (step is 1-based); returns new (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
