"""The element-wise tolerances of the surrogate's GPU parity tests, checked on
the CPU: an emulation of the device's rounding points (BF16 stores by torch's
round-to-nearest-even conversion, FP32 products and sums) must stay within the
derived tolerances of tests/bf16_bounds.py, element by element.  The
GPU tests use the same tolerances."""
import numpy as np
import pytest
import torch

from oracle import mlp as M
from tests import bf16_bounds as BB


def bf(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy()


def case(seed, n=256):
    rng = np.random.default_rng(seed)
    p = M.init_params(seed)
    for k in p:
        p[k] = p[k] + (rng.normal(0, 0.05, p[k].shape) if k in ("W4", "b4") else rng.normal(0, 0.02, p[k].shape))
    p["W4"][2:] = 0
    p["b4"][2:] = 0
    q = {k: (bf(v).astype(np.float64) if k.startswith("W") else np.float32(v).astype(np.float64)) for k, v in p.items()}
    x = bf(rng.normal(0, 1, (n, M.IN))).astype(np.float64)
    x[:, 48:] = 0
    t = rng.normal(0, 1, (n, 2))
    return q, x, t


def emulate_train(q, x, t, w_fan):
    """Forward and backward with the device's rounding points, in float32."""
    f = lambda a: np.asarray(a, np.float32)
    W = {k: f(q[f"W{k}"]) for k in (1, 2, 3, 4)}
    b = {k: f(q[f"b{k}"]) for k in (1, 2, 3, 4)}
    h = {0: f(x)}
    for k in (1, 2, 3):
        h[k] = bf(np.maximum(h[k - 1] @ W[k].T + b[k], 0))
    y = h[3] @ W[4].T + b[4]
    n = x.shape[0]
    g = {}
    pre = np.zeros_like(y)
    pre[:, 0] = (y[:, 0] - f(t[:, 0])) / np.float32(n)
    pre[:, 1] = np.float32(w_fan) * (y[:, 1] - f(t[:, 1])) / np.float32(n)
    g["b4"] = pre.sum(0)
    dy = bf(pre)
    g["W4"] = dy.T @ h[3]
    dh = dy @ W[4]
    for k in (3, 2, 1):
        v = np.where(h[k] > 0, dh, 0).astype(np.float32)
        g[f"b{k}"] = v.sum(0)
        dz = bf(v)
        g[f"W{k}"] = dz.T @ h[k - 1]
        dh = dz @ W[k]
    return y, g


@pytest.mark.parametrize("seed", [0, 1])
def test_forward_bound_covers_the_rounding_emulation(seed):
    q, x, t = case(seed)
    y_ref, sy, _, _ = BB.forward_errors(q, x)
    e_y = BB.tol(sy)
    y_em, _ = emulate_train(q, x, t, 0.5)
    err = np.abs(y_em[:, :2] - y_ref[:, :2])
    assert (err <= e_y[:, :2]).all(), (err / e_y[:, :2]).max()
    # the bound is a useful scale: well below the outputs' own size
    assert np.median(e_y[:, :2] / (np.abs(y_ref[:, :2]) + 1e-3)) < 0.15


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_bound_covers_the_rounding_emulation(seed):
    q, x, t = case(seed, n=128)
    w_fan = 0.5
    _, g_ref, eg = BB.gradient_errors(q, x, t, w_fan)
    _, g_em = emulate_train(q, x, t, w_fan)
    for name, _ in M.SHAPES:
        err = np.abs(g_em[name] - g_ref[name])
        assert (err <= eg[name] + 1e-30).all(), (name, (err / (eg[name] + 1e-30)).max())
    # the tolerances against the gradients' own scale (relative median): the
    # first layer's gradient carries the noise of three BF16 backward layers
    for name, most in (("W1", 2.0), ("W2", 0.75), ("W3", 0.3), ("W4", 0.2)):
        nz = np.abs(g_ref[name]) > 1e-12
        assert np.median(eg[name][nz] / np.abs(g_ref[name][nz])) < most, name


def test_split_first_layer_bound_covers_the_rounding_emulation():
    q, x, _ = case(3, n=512)
    x_cfg = x.copy()
    x_cfg[:, 32:] = 0
    x_inv = x.copy()
    x_inv[:, :32] = 0
    y0, e_y0 = BB.split_forward_errors(q, x_cfg, x_inv)
    f = lambda a: np.asarray(a, np.float32)
    A = bf(f(x_cfg) @ f(q["W1"]).T)
    B = bf(f(x_inv) @ f(q["W1"]).T + f(q["b1"]))
    h1 = bf(np.maximum(A + B, 0))
    h2 = bf(np.maximum(h1 @ f(q["W2"]).T + f(q["b2"]), 0))
    h3 = np.maximum(h2 @ f(q["W3"]).T + f(q["b3"]), 0)
    y_em = h3 @ f(q["W4"][0]) + f(q["b4"][0])
    err = np.abs(y_em - y0)
    assert (err <= e_y0).all(), (err / e_y0).max()
