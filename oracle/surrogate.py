"""Cost-first selection over per-invocation tables, for the learned surrogate's
decisions -- TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

When latencies and costs depend on the invocation (predicted by the
surrogate, or drawn from the ground-truth content model), every invocation i
has its own table of configurations pair_off[i] .. pair_off[i+1].  The rule is
Eq. 1's cost-first reading, written out plainly per invocation: a
configuration is feasible when its latency is strictly below the slack of its
own backend (Section 4.2); the cheapest feasible one wins, ties to the lowest
index; if none is feasible, the fastest, ties to the lowest index.
"""
from __future__ import annotations

import numpy as np


def select(lat: np.ndarray, cost: np.ndarray, slack_of_pair: np.ndarray, pair_off: np.ndarray) -> np.ndarray:
    """Chosen op-local configuration per invocation (-1 where it has no pairs)."""
    n = pair_off.shape[0] - 1
    out = np.full(n, -1, np.int64)
    for i in range(n):
        a, b = int(pair_off[i]), int(pair_off[i + 1])
        if a == b:
            continue
        L, C, S = lat[a:b], cost[a:b], slack_of_pair[a:b]
        idx = np.arange(b - a)
        feas = L < S
        if feas.any():
            f = idx[feas]
            out[i] = f[np.lexsort((f, C[feas]))[0]]
        else:
            out[i] = idx[np.lexsort((idx, L))[0]]
    return out


def forward_log_factor(params: dict, cfg_x: np.ndarray, inv_x: np.ndarray, pair_inv: np.ndarray,
                       pair_g: np.ndarray) -> np.ndarray:
    """The network's first output for (content of invocation pair_inv[k],
    configuration pair_g[k]) in float64: the inputs are the configuration's
    features in columns 0..31 and the content's in 32..47 of one row."""
    from . import mlp
    x = np.zeros((pair_inv.shape[0], mlp.IN))
    x[:, :32] = cfg_x[pair_g, :32]
    x[:, 32:48] = inv_x[pair_inv, 32:48]
    return mlp.forward(params, x)[0][:, 0]
