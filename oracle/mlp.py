"""FP64 reference of the warm-start network (test infrastructure only).

A plain numpy statement of the network the CUDA path trains and runs:
24 inputs -> 128 -> 128 (ReLU) -> 3 outputs, loss L = (1/n) sum_rows sum_c
(y - t)^2, AdamW with decoupled weight decay on the weight matrices only.
Parameters are one flat vector in the order W1 [24][128], b1 [128],
W2 [128][128], b2 [128], W3 [128][3], b3 [3] (row-major [in][out]).
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 24, 128, 3
SHAPES = [("W1", (N_IN, N_HID)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_HID, N_OUT)), ("b3", (N_OUT,))]
N_PARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(theta):
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + n], np.float64).reshape(shape)
        o += n
    return out


def flatten(p):
    return np.concatenate([np.asarray(p[name], np.float64).ravel() for name, _ in SHAPES])


def init(seed=0):
    """He-normal weights, zero biases (row-major [in][out])."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in SHAPES:
        p[name] = rng.normal(0.0, np.sqrt(2.0 / shape[0]), shape) if name[0] == "W" else np.zeros(shape)
    return flatten(p)


def forward(theta, X):
    p = unflatten(theta)
    A1 = X @ p["W1"] + p["b1"]
    H1 = np.maximum(A1, 0.0)
    A2 = H1 @ p["W2"] + p["b2"]
    H2 = np.maximum(A2, 0.0)
    Y = H2 @ p["W3"] + p["b3"]
    return Y, (X, A1, H1, A2, H2)


def loss(theta, X, T):
    Y, _ = forward(theta, X)
    return float(((Y - T) ** 2).sum() / X.shape[0])


def grad(theta, X, T):
    """Backpropagation of L = (1/n) sum (y - t)^2."""
    p = unflatten(theta)
    Y, (X, A1, H1, A2, H2) = forward(theta, X)
    n = X.shape[0]
    dY = 2.0 * (Y - T) / n
    g = {"W3": H2.T @ dY, "b3": dY.sum(0)}
    dA2 = (dY @ p["W3"].T) * (A2 > 0)
    g["W2"] = H1.T @ dA2
    g["b2"] = dA2.sum(0)
    dA1 = (dA2 @ p["W2"].T) * (A1 > 0)
    g["W1"] = X.T @ dA1
    g["b1"] = dA1.sum(0)
    return flatten(g), float(((Y - T) ** 2).sum() / n)


def is_bias_mask():
    m, o = np.zeros(N_PARAM, bool), 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        m[o:o + n] = name[0] == "b"
        o += n
    return m


def adamw(theta, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8, wd=1e-4):
    """One AdamW step (Loshchilov and Hutter): decay w <- w - lr wd w on the
    weight matrices, then w <- w - lr mhat / (sqrt(vhat) + eps)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mhat = m / (1 - b1 ** step)
    vhat = v / (1 - b2 ** step)
    decay = np.where(is_bias_mask(), 0.0, wd)
    theta = theta - lr * decay * theta
    theta = theta - lr * mhat / (np.sqrt(vhat) + eps)
    return theta, m, v
