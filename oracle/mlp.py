"""Test infrastructure, not product code: plain FP64 reference of the learned step proposer.

The network (the learned addition; the paper has no learned component) maps 12 inputs
(local position, direction, q/p, field, last step, distance to the target plane) through two
hidden layers of 64 SiLU units to one output, ln of the largest step within the RKN
tolerance. Parameters are packed as W1 [64, 12], b1 [64], W2 [64, 64], b2 [64], w3 [64],
b3 [1] (5057 values). Training minimises the mean squared error with Adam (Kingma & Ba 2015).
Only tests/ use this module; it shares no code with the CUDA kernels.
"""

from __future__ import annotations

import numpy as np

N_IN, N_HID = 12, 64
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("w3", (N_HID,)), ("b3", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)  # 5057


def unpack(theta: np.ndarray) -> dict:
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = theta[k:k + n].reshape(shape)
        k += n
    return out


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def init(seed: int) -> np.ndarray:
    """Uniform(+-1/sqrt(fan_in)) weights, zero biases."""
    rng = np.random.default_rng(seed)
    p = {"W1": rng.uniform(-1, 1, (N_HID, N_IN)) / np.sqrt(N_IN), "b1": np.zeros(N_HID),
         "W2": rng.uniform(-1, 1, (N_HID, N_HID)) / np.sqrt(N_HID), "b2": np.zeros(N_HID),
         "w3": rng.uniform(-1, 1, N_HID) / np.sqrt(N_HID), "b3": np.zeros(1)}
    return pack(p)


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def dsilu(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def forward(theta, X):
    p = unpack(np.asarray(theta, dtype=np.float64))
    z1 = X @ p["W1"].T + p["b1"]
    a1 = silu(z1)
    z2 = a1 @ p["W2"].T + p["b2"]
    a2 = silu(z2)
    out = a2 @ p["w3"] + p["b3"][0]
    return out, (X, z1, a1, z2, a2)


def bf16_round(a):
    """Values rounded to BF16 (through FP32, nearest, ties to even), returned as FP64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = (((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def loss_and_grad(theta, X, y, bf16_operands: bool = False):
    """Mean squared error over the batch and its gradient (backpropagation written out).
    With `bf16_operands` every operand of a dense contraction is rounded to BF16 first (the
    inputs and W1 for layer 1; the first activations and W2 for layer 2; dL/dZ2 and W2 for the
    backpropagation through layer 2; dL/dZ2, dL/dZ1, the first activations and the inputs for
    the weight and bias gradients), the rest stays exact: the mixed-precision training that
    runs its contractions on BF16 tensor cores."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    p = unpack(np.asarray(theta, dtype=np.float64))
    rnd = bf16_round if bf16_operands else (lambda a: a)
    Xb, W1b, W2b = rnd(X), rnd(p["W1"]), rnd(p["W2"])
    z1 = Xb @ W1b.T + p["b1"]
    a1 = silu(z1)
    a1b = rnd(a1)
    z2 = a1b @ W2b.T + p["b2"]
    a2 = silu(z2)
    out = a2 @ p["w3"] + p["b3"][0]
    n = X.shape[0]
    r = out - y
    loss = np.mean(r * r)
    dout = 2.0 * r / n
    g = {"w3": a2.T @ dout, "b3": np.array([dout.sum()])}
    dz2 = rnd(np.outer(dout, p["w3"]) * dsilu(z2))
    g["W2"] = dz2.T @ a1b
    g["b2"] = dz2.sum(0)
    dz1 = rnd((dz2 @ W2b) * dsilu(z1))
    g["W1"] = dz1.T @ Xb
    g["b1"] = dz1.sum(0)
    return loss, pack(g)


def grad_term_scale(theta, X, y):
    """For each gradient element of the BF16-operand scheme, the sum over the samples of the
    absolute values of its product terms (|dZ2|^T |A1| for W2, |dZ1|^T |X| for W1, the sums
    of |dZ| for the biases, |A2|^T |dout| and the sum of |dout| for the output layer): two
    evaluations whose BF16 operands differ by at most one unit (2^-7 of the value) differ by
    at most 2^-7 times this in that element."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    p = unpack(np.asarray(theta, dtype=np.float64))
    Xb, W1b, W2b = bf16_round(X), bf16_round(p["W1"]), bf16_round(p["W2"])
    z1 = Xb @ W1b.T + p["b1"]
    a1b = bf16_round(silu(z1))
    z2 = a1b @ W2b.T + p["b2"]
    a2 = silu(z2)
    out = a2 @ p["w3"] + p["b3"][0]
    dout = 2.0 * (out - y) / X.shape[0]
    dz2 = bf16_round(np.outer(dout, p["w3"]) * dsilu(z2))
    dz1 = bf16_round((dz2 @ W2b) * dsilu(z1))
    t = {"W1": np.abs(dz1).T @ np.abs(Xb), "b1": np.abs(dz1).sum(0), "W2": np.abs(dz2).T @ np.abs(a1b),
         "b2": np.abs(dz2).sum(0), "w3": np.abs(a2).T @ np.abs(dout), "b3": np.array([np.abs(dout).sum()])}
    return pack(t)


def adam_step(theta, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t counts from 1); returns new (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def train(theta, X, y, batch, epochs, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, bf16_operands: bool = False):
    """Mini-batches in record order (the last partial batch is dropped); returns theta and the
    mean loss of each epoch."""
    theta = np.array(theta, dtype=np.float64)
    m, v = np.zeros_like(theta), np.zeros_like(theta)
    t, losses = 0, []
    nb = X.shape[0] // batch
    for _ in range(epochs):
        acc = 0.0
        for b in range(nb):
            sl = slice(b * batch, (b + 1) * batch)
            loss, g = loss_and_grad(theta, X[sl], y[sl], bf16_operands)
            t += 1
            theta, m, v = adam_step(theta, g, m, v, t, lr, beta1, beta2, eps)
            acc += loss
        losses.append(acc / max(nb, 1))
    return theta, losses


def to_bf16(theta) -> np.ndarray:
    """Round to BF16 (nearest, ties to even); returns the 16-bit patterns."""
    f = np.asarray(theta, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return rounded.astype(np.uint16)


def from_bf16(b) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def calibrate(theta, X, y, quantile: float = 0.05):
    """The output bias shifted by the `quantile` of the residuals y - output (FP32 forward
    outputs as the library computes them are not needed here: FP64 throughout); returns the new
    parameters and the shift."""
    out, _ = forward(theta, np.asarray(X, dtype=np.float64))
    q = float(np.quantile(np.asarray(y, dtype=np.float64) - out, quantile))
    th = np.array(theta, dtype=np.float64)
    th[-1] += q
    return th, q
