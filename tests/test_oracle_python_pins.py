"""Pins of the oracle's Python functions, and mutants they must catch.

The functions pinned here judge the learned surrogate and Eq. 3's commit
order on the GPU, so each is tied to something other than itself:

* ``oracle.surrogate.select`` (Eq. 1's cost-first reading per invocation) --
  hand-derived cases (strict feasibility, per-pair slack, ties to the lowest
  index, the fastest fallback) and, on profile tables, the C oracle's
  ``or_select``, an independent implementation of the same rule;
* ``oracle.mlp.adam_step`` -- ``torch.optim.Adam`` (Kingma and Ba's update
  with bias correction, eps outside the square root) in float64;
* ``oracle.mlp.forward`` -- a hand-computed case where only a few units are
  live and every ReLU changes the answer; ``oracle.mlp.gradients`` -- torch
  autograd in float64 on the same parameters;
* ``oracle.commit_order`` (Eq. 3, Section 4.4) -- a hand-computed case:
  affinity = least objective on the other backends over the least on the
  decision's own backend, +inf when its own is 0 (1.0 when both are 0), the
  order by backend, then descending affinity, then index, invalid last.

Each mutant plants one plausible mistake in a copy of the Python source and
must fail at least one pin.
"""
import importlib.util
import math
import os

import numpy as np
import pytest

import oracle
from oracle import mlp as M
from oracle import surrogate as OS
from paper_2102_01887_b300 import workloads as W

ORACLE_DIR = os.path.dirname(oracle.__file__)


# --------------------------------------------------------------------------
# pins: each returns the names of the checks the given module fails
# --------------------------------------------------------------------------

def pin_select(mod) -> list[str]:
    failed = []
    sel = mod.select
    # hand-derived cases, one invocation each: (lat, cost, slack of each pair's backend, answer)
    cases = {
        # x0, x1, x3 feasible; x1 and x3 tie on cost 4: the lower index
        "cheapest_feasible_lowest_index": ([5, 3, 7, 3, 9], [10, 4, 4, 4, 1], [6] * 5, 1),
        # nothing feasible: the fastest, x1 and x3 tie on latency 3
        "fastest_when_none_feasible": ([5, 3, 7, 3, 9], [10, 4, 4, 4, 1], [2] * 5, 1),
        # L < slack is strict: x0 (L = slack) is infeasible although cheaper
        "strict_feasibility": ([5, 8], [1, 2], [5, 9], 1),
        # each pair against its own backend's slack
        "slack_of_own_backend": ([4, 4], [1, 2], [3, 5], 1),
        # infeasible fallback is by latency, not cost
        "fallback_by_latency": ([9, 4, 6], [1, 50, 2], [1, 1, 1], 1),
    }
    for name, (lat, cost, slk, want) in cases.items():
        got = sel(np.asarray(lat), np.asarray(cost), np.asarray(slk), np.asarray([0, len(lat)]))
        if int(got[0]) != want:
            failed.append(name)
    # an invocation without pairs
    if sel(np.zeros(0), np.zeros(0), np.zeros(0), np.asarray([0, 0, 0])).tolist() != [-1, -1]:
        failed.append("empty")
    # profile tables: the C oracle's selection (cost-first) on tie-heavy problems
    for seed in range(8):
        p, inv = W.random_small(seed, max_cfg=12, n_inv=48)
        d, _ = oracle.schedule(p, inv)
        sl = oracle.slacks(p, inv)
        valid = sl[:, 0] >= 0
        gop = p.dag_op_off[inv.dag] + inv.op_local
        sizes = np.where(valid, np.diff(p.cfg_off)[np.where(valid, gop, 0)], 0)
        off = np.concatenate([[0], np.cumsum(sizes)])
        pinv = np.repeat(np.arange(inv.n), sizes)
        px = np.arange(off[-1]) - np.repeat(off[:-1], sizes)
        pg = p.cfg_off[gop[pinv]] + px
        hw = p.hw_off.reshape(p.n_ops, p.n_hw + 1)
        lam = (hw[gop[pinv]][:, 1:p.n_hw] <= px[:, None]).sum(axis=1)
        got = sel(p.lat_us[pg], p.cost_nd[pg], sl[pinv, lam], off)
        if not np.array_equal(got[valid], d["cfg"][valid]):
            failed.append(f"c_oracle_{seed}")
    return failed


def pin_adam(mod) -> list[str]:
    import torch
    failed = []
    rng = np.random.default_rng(11)
    # a large eps so that its placement (outside the square root) matters
    for eps, lr in ((1e-3, 0.05), (0.1, 0.1)):
        p = {name: rng.normal(0, 1, shape) for name, shape in mod.SHAPES}
        m = {k: np.zeros_like(v) for k, v in p.items()}
        v = {k: np.zeros_like(x) for k, x in p.items()}
        tp = [torch.tensor(p[name].copy(), dtype=torch.float64, requires_grad=True) for name, _ in mod.SHAPES]
        opt = torch.optim.Adam(tp, lr=lr, betas=(0.9, 0.999), eps=eps)
        for step in range(1, 5):
            g = {name: rng.normal(0, 1 + step, shape) * (0.01 if step == 2 else 1.0) for name, shape in mod.SHAPES}
            mod.adam_step(p, g, m, v, step, lr, eps=eps)
            for t, (name, _) in zip(tp, mod.SHAPES):
                t.grad = torch.tensor(g[name], dtype=torch.float64)
            opt.step()
            for t, (name, _) in zip(tp, mod.SHAPES):
                if not np.allclose(p[name], t.detach().numpy(), rtol=1e-12, atol=1e-14):
                    failed.append(f"torch_adam_eps{eps}_step{step}_{name}")
                    break
    return failed


def hand_forward_params():
    """Weights with a few live units; every ReLU on the path changes the output."""
    p = {name: np.zeros(shape) for name, shape in M.SHAPES}
    p["W1"][0, 0], p["W1"][0, 1] = 1.0, 1.0  # z1[0] = 2 - 1 = 1
    p["W1"][1, 0], p["b1"][1] = -1.0, 0.5    # z1[1] = -2 + 0.5 = -1.5 -> 0
    p["b1"][2] = 0.25                        # z1[2] = 0.25
    p["W2"][0, 0] = 3.0                      # z2[0] = 3 * h1[0] = 3
    p["W2"][0, 1] = 100.0                    # h1[1] = 0: nothing (a missing ReLU gives -150)
    p["W2"][1, 2] = -4.0                     # z2[1] = -4 * 0.25 = -1 -> 0
    p["W3"][0, 0], p["W3"][0, 1] = 0.5, 7.0  # z3[0] = 1.5 + 7 * h2[1] = 1.5
    p["b3"][1] = -2.0                        # z3[1] = -2 -> 0
    p["W4"][0, 0], p["W4"][0, 1] = 2.0, 9.0  # y0 = 2 * 1.5 + 9 * h3[1] + 0.125 = 3.125
    p["b4"][0] = 0.125
    p["W4"][1, 0], p["b4"][1] = -1.0, 0.5    # y1 = -1.5 + 0.5 = -1.0 (no ReLU on the output)
    p["b4"][5] = -0.75                       # an output row the loss never reads, unclipped
    x = np.zeros((1, M.IN))
    x[0, 0], x[0, 1] = 2.0, -1.0
    return p, x


def pin_forward(mod) -> list[str]:
    import torch
    failed = []
    p, x = hand_forward_params()
    y, _ = mod.forward(p, x)
    want = np.zeros(M.OUT)
    want[0], want[1], want[5] = 3.125, -1.0, -0.75
    if not np.allclose(y[0], want, rtol=0, atol=1e-12):
        failed.append("hand_forward")
    # gradients against torch autograd in float64
    rng = np.random.default_rng(5)
    q = M.init_params(2)
    for name in q:
        q[name] = q[name] + rng.normal(0, 0.05, q[name].shape)
    xs = rng.normal(0, 1, (9, M.IN))
    ts = rng.normal(0, 1, (9, 2))
    w_fan = 0.3
    lv, g = mod.gradients(q, xs, ts, w_fan)
    tq = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in q.items()}
    h = torch.tensor(xs, dtype=torch.float64)
    for k in (1, 2, 3):
        h = torch.relu(torch.nn.functional.linear(h, tq[f"W{k}"], tq[f"b{k}"]))
    yt = torch.nn.functional.linear(h, tq["W4"], tq["b4"])
    tt = torch.tensor(ts, dtype=torch.float64)
    lt = (0.5 * (yt[:, 0] - tt[:, 0]) ** 2 + 0.5 * w_fan * (yt[:, 1] - tt[:, 1]) ** 2).mean()
    lt.backward()
    if not math.isclose(lv, float(lt.detach()), rel_tol=1e-12):
        failed.append("autograd_loss")
    for name, _ in M.SHAPES:
        if not np.allclose(g[name], tq[name].grad.numpy(), rtol=1e-10, atol=1e-14):
            failed.append(f"autograd_{name}")
    return failed


def commit_case():
    """Seven decided invocations of the tiny workload (backends of 8 configurations
    each) with chosen per-backend minima."""
    p, inv = W.tiny()
    sub = inv.subset(np.arange(7))
    dec = np.zeros(7, dtype=oracle.DECISION_DTYPE)
    dec["cfg"] = [0, 3, 7, 8, -1, 2, 5]  # backends 0, 0, 0, 1, invalid, 0, 0
    dec["flags"] = [1, 1, 0, 1, oracle.FLAG_INVALID, 1, 1]
    big = 2**63 - 1
    obj = np.asarray([[10, 30, 20],   # own 10, others min(30, 20) = 20 -> 2.0
                      [0, 5, 7],      # own 0 -> +inf
                      [40, 10, 80],   # 10 / 40 = 0.25
                      [5, 20, 15],    # backend 1: own 20, others min(5, 15) = 5 -> 0.25
                      [big, big, big],
                      [0, 0, 3],      # own 0 and others 0 -> 1.0
                      [8, 16, 50]],   # 16 / 8 = 2.0, ties with invocation 0
                     np.int64)
    order = [1, 0, 6, 5, 2, 3, 4]
    aff = [2.0, math.inf, 0.25, 0.25, 0.0, 1.0, 2.0]
    return p, sub, dec, obj, order, aff


def pin_commit(mod) -> list[str]:
    failed = []
    p, sub, dec, obj, order, aff = commit_case()
    got_order, got_aff = mod.commit_order(p, sub, dec, obj)
    if got_order.tolist() != order:
        failed.append("hand_order")
    if got_aff.tolist() != aff:
        failed.append("hand_affinity")
    return failed


PINS = {"surrogate": pin_select, "mlp_adam": pin_adam, "mlp_forward": pin_forward, "commit": pin_commit}
SOURCES = {"surrogate": "surrogate.py", "mlp_adam": "mlp.py", "mlp_forward": "mlp.py", "commit": "__init__.py"}
REAL = {"surrogate": OS, "mlp_adam": M, "mlp_forward": M, "commit": oracle}


@pytest.mark.parametrize("which", sorted(PINS))
def test_oracle_function_passes_its_pins(which):
    assert PINS[which](REAL[which]) == []


MUTANTS = {
    # surrogate.select
    "select_not_strict": ("surrogate", "feas = L < S", "feas = L <= S"),
    "select_fallback_cheapest": ("surrogate", "out[i] = idx[np.lexsort((idx, L))[0]]",
                                 "out[i] = idx[np.lexsort((idx, C))[0]]"),
    "select_ties_highest_index": ("surrogate", "out[i] = f[np.lexsort((f, C[feas]))[0]]",
                                  "out[i] = f[np.lexsort((-f, C[feas]))[0]]"),
    "select_first_pair_slack": ("surrogate", "L, C, S = lat[a:b], cost[a:b], slack_of_pair[a:b]",
                                "L, C, S = lat[a:b], cost[a:b], np.full(b - a, slack_of_pair[a])"),
    # mlp.adam_step
    "adam_no_bias_correction": ("mlp_adam", "mh = m[name] / (1 - b1 ** step)", "mh = m[name]"),
    "adam_no_second_correction": ("mlp_adam", "vh = v[name] / (1 - b2 ** step)", "vh = v[name]"),
    "adam_eps_inside_sqrt": ("mlp_adam", "np.sqrt(vh) + eps", "np.sqrt(vh + eps)"),
    "adam_step_off_by_one": ("mlp_adam", "(1 - b1 ** step)", "(1 - b1 ** (step + 1))"),
    "adam_first_moment_of_square": ("mlp_adam", "(1 - b2) * g[name] ** 2", "(1 - b2) * abs(g[name])"),
    # mlp.forward / gradients
    "forward_missing_relu_layer1": ("mlp_forward", "h1 = np.maximum(z1, 0.0)", "h1 = z1"),
    "forward_missing_relu_layer2": ("mlp_forward", "h2 = np.maximum(z2, 0.0)", "h2 = z2"),
    "forward_missing_relu_layer3": ("mlp_forward", "h3 = np.maximum(z3, 0.0)", "h3 = z3"),
    "forward_relu_on_output": ("mlp_forward", 'y = h3 @ p["W4"].T + p["b4"]',
                               'y = np.maximum(h3 @ p["W4"].T + p["b4"], 0.0)'),
    "forward_transposed_w2": ("mlp_forward", 'z2 = h1 @ p["W2"].T + p["b2"]', 'z2 = h1 @ p["W2"] + p["b2"]'),
    "gradients_wrong_mask": ("mlp_forward", 'dz2 = (dz3 @ p["W3"]) * (z2 > 0)', 'dz2 = (dz3 @ p["W3"]) * (z3 > 0)'),
    "gradients_drop_fan_weight": ("mlp_forward", 'dy[:, 1] = w_fan * (y[:, 1] - t[:, 1]) / n',
                                  'dy[:, 1] = (y[:, 1] - t[:, 1]) / n'),
    # commit_order (Eq. 3)
    "commit_inverted_affinity": ("commit", "else float(other) / float(own)", "else float(own) / float(other)"),
    "commit_zero_own_is_zero": ("commit", '(1.0 if other == 0 else float("inf")) if own == 0',
                                "0.0 if own == 0"),
    "commit_ascending_affinity": ("commit", "keys.append((lam, -a, i))", "keys.append((lam, a, i))"),
    "commit_other_is_max": ("commit", "other = min(int(obj_min[i, h])", "other = max(int(obj_min[i, h])"),
}


def load_mutant(which: str, old: str, new: str, tmp_path):
    src_path = os.path.join(ORACLE_DIR, SOURCES[which])
    src = open(src_path).read()
    assert src.count(old) == 1, f"mutation site not unique: {old}"
    path = tmp_path / f"mutant_{which}.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location(f"oracle_mutant_{which}", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_python_mutant_is_caught(name, tmp_path):
    which, old, new = MUTANTS[name]
    mod = load_mutant(which, old, new, tmp_path)
    failed = PINS[which](mod)
    assert failed, f"mutant {name} passed every pin of {which}"
