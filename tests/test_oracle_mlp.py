"""Pins of the surrogate network's FP64 oracle: its analytic gradients against
central finite differences of its own loss, a closed form, and invariants."""
import numpy as np
import pytest

from oracle import mlp as M


def small_case(seed, n=7):
    rng = np.random.default_rng(seed)
    p = M.init_params(seed)
    for name in p:  # nonzero biases and output rows so every term matters
        p[name] = p[name] + rng.normal(0, 0.05, p[name].shape)
    x = rng.normal(0, 1, (n, M.IN))
    t = rng.normal(0, 1, (n, 2))
    return p, x, t


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradients_match_central_differences(seed):
    p, x, t = small_case(seed)
    w_fan = 0.7
    _, g = M.gradients(p, x, t, w_fan)
    rng = np.random.default_rng(100 + seed)
    h = 1e-6
    for name, shape in M.SHAPES:
        for _ in range(6):
            idx = tuple(int(rng.integers(0, s)) for s in shape)
            q = {k: v.copy() for k, v in p.items()}
            q[name][idx] += h
            lp = M.loss(M.forward(q, x)[0], t, w_fan)
            q[name][idx] -= 2 * h
            lm = M.loss(M.forward(q, x)[0], t, w_fan)
            fd = (lp - lm) / (2 * h)
            assert abs(g[name][idx] - fd) <= 1e-6 + 1e-5 * abs(fd), (name, idx, g[name][idx], fd)


def test_output_layer_closed_form():
    # with all hidden activations known, dW4 = dy^T h3 and db4 = sum dy exactly
    p, x, t = small_case(5, n=11)
    _, g = M.gradients(p, x, t, 1.0)
    y, cache = M.forward(p, x)
    h3 = cache[-1]
    dy = np.zeros_like(y)
    dy[:, :2] = (y[:, :2] - t) / x.shape[0]
    for i in range(M.OUT):
        for j in (0, 17, 255):
            assert g["W4"][i, j] == pytest.approx(sum(dy[k, i] * h3[k, j] for k in range(x.shape[0])), abs=1e-12)
    assert np.allclose(g["b4"][:2], dy[:, :2].sum(0))
    assert not g["W4"][2:].any() and not g["b4"][2:].any()  # rows the loss never reads


def test_dead_units_get_no_gradient():
    p, x, t = small_case(9)
    p["b1"][:] = -1e3  # every first-layer unit is off: nothing reaches W1, b1, nor W2 (h1 = 0)
    _, g = M.gradients(p, x, t, 1.0)
    for name in ("W1", "b1", "W2"):
        assert not g[name].any(), name
    assert g["W3"].any()  # layer 2 still passes its biases on


def test_pack_roundtrip_and_count():
    p = M.init_params(3)
    flat = M.pack(p)
    assert flat.shape == (M.N_PARAMS,) == (164672,)
    q = M.unpack(flat)
    assert all(np.array_equal(p[k], q[k]) for k in p)


def test_adam_moves_against_the_gradient():
    p, x, t = small_case(4)
    l0, g = M.gradients(p, x, t, 1.0)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(v) for k, v in p.items()}
    for step in range(1, 30):
        _, g = M.gradients(p, x, t, 1.0)
        M.adam_step(p, g, m, v, step, 1e-3)
    assert M.gradients(p, x, t, 1.0)[0] < l0
