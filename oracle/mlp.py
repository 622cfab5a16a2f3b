"""FP64 CPU oracle of the proposal network — TEST INFRASTRUCTURE.

A 12 -> 64 -> 64 -> 1 multilayer perceptron with ReLU scores each candidate
partner of a site from 12 pair features; a site's candidates compete through a
softmax (listwise).  Training minimises the cross-entropy of the partner that
actually formed a bond in a plain (DyBond) run.  This module is the plain
NumPy definition in float64 that the tensor-core kernels are checked against;
its backward pass is pinned by central finite differences in the tests.

Parameter layout (float32 on the device, float64 here), in this order:
W1[16][64] (rows 12..15 unused, zero), b1[64], W2[64][64], b2[64], w3[64], b3[1].
"""
from __future__ import annotations

import numpy as np

NF = 12          # features per candidate
KPAD = 16        # padded input width
H = 64           # hidden width
SIZES = [("W1", (KPAD, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))]
NPARAM = sum(int(np.prod(s)) for _, s in SIZES)


def unpack(theta):
    out, o = {}, 0
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def init(seed=0, scale=1.0):
    """He-style initial weights (what the device training starts from too)."""
    rng = np.random.default_rng(seed)
    p = {"W1": np.zeros((KPAD, H)), "b1": np.zeros(H), "W2": rng.normal(0, np.sqrt(2 / H), (H, H)) * scale,
         "b2": np.zeros(H), "w3": rng.normal(0, np.sqrt(1 / H), H) * scale, "b3": np.zeros(1)}
    p["W1"][:NF] = rng.normal(0, np.sqrt(2 / NF), (NF, H)) * scale
    return pack(p)


def forward(theta, X):
    """X: (rows, 12 or 16) -> logits (rows,) and the cache for backward."""
    p = unpack(theta)
    Xp = np.zeros((X.shape[0], KPAD))
    Xp[:, :X.shape[1]] = X
    Z1 = Xp @ p["W1"] + p["b1"]
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ p["W2"] + p["b2"]
    H2 = np.maximum(Z2, 0.0)
    y = H2 @ p["w3"] + p["b3"][0]
    return y, (Xp, Z1, H1, Z2, H2)


def listwise_loss(y, offsets, labels):
    """Mean over events of -log softmax(y[event])[label]; offsets has E+1
    entries delimiting each event's candidate rows.  Returns (loss, dL/dy)."""
    E = len(labels)
    dy = np.zeros_like(y)
    loss = 0.0
    for e in range(E):
        a, b = offsets[e], offsets[e + 1]
        z = y[a:b] - y[a:b].max()
        pz = np.exp(z) / np.exp(z).sum()
        loss -= np.log(pz[labels[e]])
        g = pz.copy()
        g[labels[e]] -= 1.0
        dy[a:b] = g / E
    return loss / E, dy


def backward(theta, cache, dy):
    """Gradient of sum(dy * y) with respect to the packed parameters."""
    p = unpack(theta)
    Xp, Z1, H1, Z2, H2 = cache
    g = {}
    g["w3"] = H2.T @ dy
    g["b3"] = np.array([dy.sum()])
    dZ2 = np.outer(dy, p["w3"]) * (Z2 > 0)
    g["W2"] = H1.T @ dZ2
    g["b2"] = dZ2.sum(0)
    dZ1 = (dZ2 @ p["W2"].T) * (Z1 > 0)
    g["W1"] = Xp.T @ dZ1
    g["W1"][NF:] = 0.0
    g["b1"] = dZ1.sum(0)
    return pack(g)


def loss_and_grad(theta, X, offsets, labels):
    y, cache = forward(theta, X)
    loss, dy = listwise_loss(y, offsets, labels)
    return loss, backward(theta, cache, dy)


def adam_step(theta, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(a):
    """Round float values to bfloat16 (round to nearest even) and back."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def forward_bf16(theta, X):
    """Forward pass with the operands of both matrix products rounded to
    BF16 as a BF16 tensor-core evaluation takes them (inputs, W1, W2 and the
    first hidden layer); biases, w3 and every sum exact in FP64."""
    p = unpack(theta)
    rb = lambda a: bf16_round(a).astype(np.float64)
    Xp = np.zeros((X.shape[0], KPAD))
    Xp[:, :X.shape[1]] = X
    Xb, W1b, W2b = rb(Xp), rb(p["W1"]), rb(p["W2"])
    Z1 = Xb @ W1b + p["b1"]
    H1b = rb(np.maximum(Z1, 0.0))
    Z2 = H1b @ W2b + p["b2"]
    H2 = np.maximum(Z2, 0.0)
    y = H2 @ p["w3"] + p["b3"][0]
    return y, (Xb, W2b, Z1, H1b, Z2, H2)


def loss_and_grad_bf16(theta, X, offsets, labels):
    """Loss and gradient of forward_bf16 with the back-propagated dZ2 and dZ1
    rounded to BF16 as well (the operands of the backward products); the
    listwise loss and every sum exact in FP64.  It is the reference for what
    BF16 operands alone cost in accuracy: a device evaluation differs from it
    only by its FP32 summation order."""
    p = unpack(theta)
    rb = lambda a: bf16_round(a).astype(np.float64)
    y, (Xb, W2b, Z1, H1b, Z2, H2) = forward_bf16(theta, X)
    loss, dy = listwise_loss(y, offsets, labels)
    g = {}
    g["w3"] = H2.T @ dy
    g["b3"] = np.array([dy.sum()])
    dZ2b = rb(np.outer(dy, p["w3"]) * (Z2 > 0))
    g["W2"] = H1b.T @ dZ2b
    g["b2"] = dZ2b.sum(0)
    dZ1b = rb((dZ2b @ W2b.T) * (Z1 > 0))
    g["W1"] = Xb.T @ dZ1b
    g["W1"][NF:] = 0.0
    g["b1"] = dZ1b.sum(0)
    return loss, y, pack(g)
