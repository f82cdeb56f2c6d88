"""Plain NumPy FP64 statement of the latency surrogate's network -- TEST
INFRASTRUCTURE, like the rest of ``oracle/``: only the tests, the smoke check
and the benchmark's CPU legs use it; the product path never does.

The network: input of 64 features (48 used, zero padding), three hidden
layers of width 256 with ReLU, a linear output layer of 64 rows of which the
first two are read (log latency factor, branch fan-out).  Loss: the mean over
the batch of (y0 - t0)^2 / 2 + w_fan (y1 - t1)^2 / 2.

The gradients are the chain rule written out layer by layer (a linear layer
z = h W^T + b has dW = dz^T h, db = sum of dz over the batch, dh = dz W; a ReLU
passes dz where its input was positive).  The flat parameter order matches the
C ABI: W1[256x64], b1[256], W2[256x256], b2, W3[256x256], b3, W4[64x256], b4[64].
"""
from __future__ import annotations

import numpy as np

IN, HID, OUT = 64, 256, 64
SHAPES = [("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (HID, HID)), ("b3", (HID,)), ("W4", (OUT, HID)), ("b4", (OUT,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def init_params(seed: int = 0) -> dict:
    """He-uniform hidden layers, a small output layer, zero biases (float64)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in SHAPES:
        if name.startswith("b"):
            p[name] = np.zeros(shape)
        else:
            fan_in = shape[1]
            lim = np.sqrt(6.0 / fan_in) * (0.1 if name == "W4" else 1.0)
            p[name] = rng.uniform(-lim, lim, shape)
    p["W4"][2:] = 0.0
    p["b4"][2:] = 0.0
    return p


def pack(p: dict) -> np.ndarray:
    return np.concatenate([np.asarray(p[n], np.float64).ravel() for n, _ in SHAPES])


def unpack(flat: np.ndarray) -> dict:
    p, o = {}, 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        p[name] = np.asarray(flat[o:o + k], np.float64).reshape(shape)
        o += k
    return p


def pad_features(x: np.ndarray) -> np.ndarray:
    out = np.zeros((x.shape[0], IN))
    out[:, :x.shape[1]] = x
    return out


def forward(p: dict, x: np.ndarray):
    """Outputs float64[n, 64] and the activations the backward pass needs."""
    h0 = np.asarray(x, np.float64)
    z1 = h0 @ p["W1"].T + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ p["W3"].T + p["b3"]
    h3 = np.maximum(z3, 0.0)
    y = h3 @ p["W4"].T + p["b4"]
    return y, (h0, z1, h1, z2, h2, z3, h3)


def loss(y: np.ndarray, t: np.ndarray, w_fan: float) -> float:
    n = y.shape[0]
    return float((0.5 * (y[:, 0] - t[:, 0]) ** 2 + 0.5 * w_fan * (y[:, 1] - t[:, 1]) ** 2).sum() / n)


def gradients(p: dict, x: np.ndarray, t: np.ndarray, w_fan: float):
    """(loss, gradient dict) of the mean loss over the batch."""
    y, (h0, z1, h1, z2, h2, z3, h3) = forward(p, x)
    n = y.shape[0]
    dy = np.zeros_like(y)
    dy[:, 0] = (y[:, 0] - t[:, 0]) / n
    dy[:, 1] = w_fan * (y[:, 1] - t[:, 1]) / n
    g = {"W4": dy.T @ h3, "b4": dy.sum(0)}
    dz3 = (dy @ p["W4"]) * (z3 > 0)
    g["W3"], g["b3"] = dz3.T @ h2, dz3.sum(0)
    dz2 = (dz3 @ p["W3"]) * (z2 > 0)
    g["W2"], g["b2"] = dz2.T @ h1, dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * (z1 > 0)
    g["W1"], g["b1"] = dz1.T @ h0, dz1.sum(0)
    return loss(y, t, w_fan), g


def adam_step(p: dict, g: dict, m: dict, v: dict, step: int, lr: float, b1: float = 0.9,
              b2: float = 0.999, eps: float = 1e-8) -> None:
    """One Adam update in place (Kingma and Ba, 2015), step counted from 1."""
    for name, _ in SHAPES:
        m[name] = b1 * m[name] + (1 - b1) * g[name]
        v[name] = b2 * v[name] + (1 - b2) * g[name] ** 2
        mh = m[name] / (1 - b1 ** step)
        vh = v[name] / (1 - b2 ** step)
        p[name] = p[name] - lr * mh / (np.sqrt(vh) + eps)
