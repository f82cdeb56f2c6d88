"""Element-wise tolerances for the surrogate network computed in BF16 with FP32
accumulation, against the FP64 oracle (oracle/mlp.py) on the same BF16-rounded
inputs and weights.

Probabilistic rounding error analysis (Higham and Mary, "A new approach to
probabilistic rounding error analysis", SIAM J. Sci. Comput. 41(5), 2019):
rounding errors are modelled as independent, mean-zero, bounded by u|v| at
each rounding point, so the error of a K-term sum of perturbed terms grows like
the square root of the sum of the terms' variances, not like the sum of their
bounds (which would make a worst-case bound grow ~sqrt(K) times faster per
layer and exceed the outputs themselves after three layers of width 256).
Every quantity v the device computes carries the variance s2 of its rounding
error, propagated in quadrature:

* a BF16 store of v adds (u |v|)^2, u = 2^-8 (8-bit significand, round to
  nearest; a uniform error on [-u|v|, u|v|] has variance (u|v|)^2 / 3, so this
  is conservative), an FP32 store (2^-24 |v|)^2;
* a product-sum z_j = sum_k a_jk b_k of K terms adds
  sum_k (b_k^2 s2(a_jk) + a_jk^2 s2(b_k)) from its operands, and
  K (2^-24 sum_k |a_jk b_k|)^2 from its FP32 accumulation (at most K
  roundings, each within 2^-24 of a partial sum);
* ReLU is 1-Lipschitz and passes s2 through in the forward pass; in the
  backward pass a ReLU mask of the device differs from the oracle's where the
  device's z has the other sign, with probability Phi(-|z| / sigma(z)) under a
  Gaussian model; the masked gradient then differs by the whole incoming
  gradient g, a rare, sign-random term of variance p g^2 in the later sums.

The tolerance of an element is LAMBDA sigma, LAMBDA = 8 (a Gaussian tail
beyond 8 sigma has probability about 1e-15 per element).

Where the device rounds (paper_2102_01887_b300/csrc/sg_mlp.cu, sg_gemm.cu):
training forward -- h1, h2, h3 stored BF16 after the FP32 bias and the ReLU,
y in FP32; backward -- dy stored BF16, the ReLU-masked dh stored BF16 (dz)
while the bias gradient sums the unrounded FP32 values; scheduling -- the split
first layer's configuration part A stored BF16, the content part B (with b1)
rounded to BF16, h1 = ReLU(A + B) rounded once, h2 in BF16, h3 kept in FP32 and
folded with the FP32 last-layer row.

The intermediates come from the oracle (forward caches; per-sample dz from the
oracle's bias gradients of one-sample batches), so these are scales for
comparing the device with the oracle, not a second statement of the network.
tests/test_bf16_bounds.py checks them on the CPU against an emulation of the
device's rounding points.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erfc

from oracle import mlp as M

U16 = 2.0 ** -8
U32 = 2.0 ** -24
LAMBDA = 8.0


def tol(s2):
    return LAMBDA * np.sqrt(s2)


def store(v, s2, u=U16):
    """Variance after storing v (already within variance s2) with unit roundoff u."""
    return s2 + (u * np.abs(v)) ** 2


def product(a, sa, b, sb):
    """Variance of the FP32 product a @ b from operands with variances sa, sb."""
    k = a.shape[-1]
    acc = np.abs(a) @ np.abs(b)
    return (a * a) @ sb + sa @ (b * b) + k * (U32 * acc) ** 2


def linear(h, sh, W, b):
    """z = h W^T + b with exact weights, the bias added in FP32."""
    s2 = product(h, sh, W.T, np.zeros(W.T.shape))
    return s2 + (U32 * (np.abs(h) @ np.abs(W).T + np.abs(b))) ** 2


def forward_errors(q: dict, x: np.ndarray):
    """Training-path forward: (y, variance of y, oracle cache, variances of z1..z3, h1..h3)."""
    y, cache = M.forward(q, x)
    h0, z1, h1, z2, h2, z3, h3 = cache
    e = {"z1": linear(h0, np.zeros_like(h0), q["W1"], q["b1"])}
    e["h1"] = store(h1, e["z1"])
    e["z2"] = linear(h1, e["h1"], q["W2"], q["b2"])
    e["h2"] = store(h2, e["z2"])
    e["z3"] = linear(h2, e["h2"], q["W3"], q["b3"])
    e["h3"] = store(h3, e["z3"])
    sy = store(y, linear(h3, e["h3"], q["W4"], q["b4"]), U32)
    return y, sy, cache, e


def per_sample_dz(q: dict, x: np.ndarray, t: np.ndarray, w_fan: float):
    """dz_k of every sample for the batch-mean loss, from the oracle's bias
    gradients of one-sample batches (divided by the batch size)."""
    n = x.shape[0]
    dz = {k: np.zeros((n, M.HID)) for k in (1, 2, 3)}
    for i in range(n):
        _, g = M.gradients(q, x[i:i + 1], t[i:i + 1], w_fan)
        for k in (1, 2, 3):
            dz[k][i] = g[f"b{k}"] / n
    return dz


def flip_probability(z, sz):
    """Probability that the device's z has the other sign than the oracle's."""
    sig = np.sqrt(sz)
    return np.where(sig > 0, 0.5 * erfc(np.abs(z) / (np.sqrt(2.0) * np.maximum(sig, 1e-300))),
                    (z == 0).astype(float))


def gradient_errors(q: dict, x: np.ndarray, t: np.ndarray, w_fan: float):
    """(loss, oracle gradients, tolerance per gradient element) of the training path."""
    n = x.shape[0]
    loss, g = M.gradients(q, x, t, w_fan)
    y, sy, cache, ef = forward_errors(q, x)
    h0, z1, h1, z2, h2, z3, h3 = cache
    hs = {0: h0, 1: h1, 2: h2, 3: h3}
    shs = {0: np.zeros_like(h0), 1: ef["h1"], 2: ef["h2"], 3: ef["h3"]}
    zs = {1: z1, 2: z2, 3: z3}
    dz = per_sample_dz(q, x, t, w_fan)
    w = np.asarray([1.0, w_fan])
    dy = np.zeros((n, M.OUT))
    dy[:, :2] = (y[:, :2] - t) * w / n
    pre = np.zeros_like(dy)  # (y - t) w / n in FP32, before the BF16 store
    pre[:, :2] = store(dy[:, :2], sy[:, :2] * (w / n) ** 2, 2 * U32)
    sdy = store(dy, pre)
    sdy[:, 2:] = 0.0
    out = {"b4": tol(pre.sum(0) + n * (U32 * np.abs(dy).sum(0)) ** 2)}
    out["W4"] = tol(product(dy.T, sdy.T, h3, shs[3]))
    dh = dy @ q["W4"]
    sdh = product(dy, sdy, q["W4"], np.zeros(q["W4"].shape))
    for k in (3, 2, 1):
        v = dz[k]
        live = zs[k] > 0
        sv = np.where(live, sdh, 0.0) + flip_probability(zs[k], ef[f"z{k}"]) * (np.abs(dh) + tol(sdh)) ** 2
        out[f"b{k}"] = tol(sv.sum(0) + n * (U32 * np.abs(v).sum(0)) ** 2)
        sdz = store(v, sv)
        out[f"W{k}"] = tol(product(v.T, sdz.T, hs[k - 1], shs[k - 1]))
        if k > 1:
            dh = v @ q[f"W{k}"]
            sdh = product(v, sdz, q[f"W{k}"], np.zeros(q[f"W{k}"].shape))
    return loss, g, out


def split_forward_errors(q: dict, x_cfg: np.ndarray, x_inv: np.ndarray):
    """Scheduling path: the log latency factor y0 of pairs whose first-layer
    inputs are x_cfg (configuration columns, others 0) and x_inv (content
    columns), and its tolerance."""
    A = x_cfg @ q["W1"].T
    B = x_inv @ q["W1"].T + q["b1"]
    sA = store(A, linear(x_cfg, np.zeros_like(x_cfg), q["W1"], np.zeros(M.HID)))
    sB = store(B, linear(x_inv, np.zeros_like(x_inv), q["W1"], q["b1"]))
    y, cache = M.forward(q, x_cfg + x_inv)
    _, z1, h1, z2, h2, z3, h3 = cache
    sh1 = store(h1, sA + sB)  # A + B rounded once (fused add and ReLU)
    sh2 = store(h2, linear(h1, sh1, q["W2"], q["b2"]))
    sh3 = store(h3, linear(h2, sh2, q["W3"], q["b3"]), U32)  # kept in FP32
    sy0 = linear(h3, sh3, q["W4"][:1], q["b4"][:1])
    return y[:, 0], tol(sy0)[:, 0]
