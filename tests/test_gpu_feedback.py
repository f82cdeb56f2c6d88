"""Queueing time (Eq. 2) on the device, and exponential-smoothing feedback that
updates the tables in place (Section 3.3): tables and later decisions bit-exact
against the oracle applying the same integer rules."""
import copy

import numpy as np
import pytest

import oracle
from paper_2102_01887_b300 import workloads as W

pytestmark = pytest.mark.gpu
FIELDS = ("cfg", "lat", "cost", "slack", "flags")


@pytest.fixture(scope="module")
def L(cuda_device):
    from paper_2102_01887_b300 import build, llama
    build.build()
    llama.load()
    return llama


def same(a, b, what=""):
    for f in FIELDS:
        bad = np.flatnonzero(a[f] != b[f])
        assert bad.size == 0, f"{what} {f}: {bad.size} mismatches at {bad[:5]}"


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("method", [0, 1], ids=["scan", "staircase"])
def test_queue_time_feeds_the_next_call(L, method):
    import torch
    p, inv = W.medium()
    p.q_us = np.zeros(p.n_hw, np.int64)
    queued = inv.subset(np.arange(0, inv.n, 3))
    later = inv.subset(np.arange(1, inv.n, 3))
    with L.Scheduler(p, method=method, use_graph=True) as s:
        d_q, _ = s.schedule(queued)
        q = torch.zeros(p.n_hw, dtype=torch.int64, device="cuda")
        dec = dev(d_q.view(np.uint8))
        L.llama_queue_time(s.ctx, dev(queued.dag), dev(queued.op_local), dec, q, apply=True)
        got_q = q.cpu().numpy()
        d_later, _ = s.schedule(later)
    exp_q = oracle.queue_time(p, queued, d_q)
    assert np.array_equal(got_q, exp_q) and (exp_q > 0).any()
    p2 = copy.deepcopy(p)
    p2.q_us = exp_q
    exp, _ = oracle.schedule(p2, later)
    same(d_later, exp, "after Eq. 2")


@pytest.mark.parametrize("mode,alpha", [(0, (1, 1)), (1, (3, 2))], ids=["cost_first", "alpha"])
@pytest.mark.parametrize("method", [0, 1], ids=["scan", "staircase"])
def test_feedback_updates_tables_and_decisions(L, mode, alpha, method):
    p, inv = W.medium()
    rng = np.random.default_rng(7)
    n = 40_000
    hot = rng.integers(0, p.n_cfg, 3000)  # repeated configurations: the order matters
    g = hot[rng.integers(0, hot.shape[0], n)]
    op = (np.searchsorted(p.cfg_off, g, side="right") - 1).astype(np.int32)
    cfg = (g - p.cfg_off[op]).astype(np.int32)
    lat = np.maximum(1, p.lat_us[g] * rng.uniform(0.3, 3.0, n)).astype(np.int32)
    cost = (p.cost_nd[g] * rng.uniform(0.5, 2.0, n)).astype(np.int64)
    op[:3], cfg[3:5], lat[5] = -1, 10**6, 0  # six invalid observations
    sub = inv.subset(np.arange(0, inv.n, 4))
    with L.Scheduler(p, mode=mode, alpha=alpha, method=method, use_graph=True) as s:
        before, _ = s.schedule(sub)  # captures the graph that must see the new tables
        import torch
        rej = torch.zeros(1, dtype=torch.int64, device="cuda")
        L.llama_feedback(s.ctx, dev(op), dev(cfg), dev(lat), dev(cost), beta=(1, 4), rejected=rej)
        after, _ = s.schedule(sub)
        lat_d, cost_d = L.llama_get_profiles(s.ctx, p.n_cfg)
        n_rej = int(rej.item())
    q = copy.deepcopy(p)
    exp_rej = oracle.feedback(q, op, cfg, lat, cost, beta=(1, 4))
    assert n_rej == exp_rej == 6
    assert np.array_equal(lat_d, q.lat_us) and np.array_equal(cost_d, q.cost_nd)
    exp, _ = oracle.schedule(q, sub, mode=mode, alpha=alpha)
    same(after, exp, "after feedback")
    assert (after["cfg"] != before["cfg"]).any()


@pytest.mark.parametrize("count_pass", [1, 2], ids=["count_pass_on", "count_pass_off"])
def test_feedback_on_tables_beyond_the_staged_latencies(L, count_pass):
    # 8,192-configuration ops: the feedback re-encodes the touched ops' distinct
    # latencies and both levels of probe lines, which the count pass (or, with
    # it off, the scoring kernel's own searches) reads on the next call
    p, inv = W.batched_large(n_dags=8, n_inv=4096)
    rng = np.random.default_rng(11)
    n = 20_000
    ops = np.unique(p.dag_op_off[inv.dag] + inv.op_local)[:120]  # invoked ops
    g = np.concatenate([rng.integers(p.cfg_off[v], p.cfg_off[v + 1], 100) for v in ops])
    g = g[rng.integers(0, g.shape[0], n)]
    op = (np.searchsorted(p.cfg_off, g, side="right") - 1).astype(np.int32)
    cfg = (g - p.cfg_off[op]).astype(np.int32)
    # faster and cheaper than profiled: about a third of the decisions change
    lat = np.maximum(1, p.lat_us[g] * rng.uniform(0.05, 0.5, n)).astype(np.int32)
    cost = (p.cost_nd[g] * rng.uniform(0.1, 0.5, n)).astype(np.int64)
    with L.Scheduler(p, use_graph=True) as s:
        L.llama_set_count_pass(s.ctx, count_pass)
        before, _ = s.schedule(inv)
        L.llama_feedback(s.ctx, dev(op), dev(cfg), dev(lat), dev(cost), beta=(1, 2))
        after, _ = s.schedule(inv)
        assert L.llama_last_launch_count(s.ctx) == (3 if count_pass == 1 else 2)
    q = copy.deepcopy(p)
    assert oracle.feedback(q, op, cfg, lat, cost, beta=(1, 2)) == 0
    exp, _ = oracle.schedule(q, inv)
    same(after, exp, "after feedback")
    assert (after["cfg"] != before["cfg"]).sum() > 1000


@pytest.mark.parametrize("method", [0, 1], ids=["scan", "staircase"])
def test_affinity_and_commit_order(L, method):
    import torch
    p, inv = W.medium()
    sub = inv.subset(np.arange(0, inv.n, 160))  # 410 invocations
    sub.dag = sub.dag.copy()
    sub.dag[4] = -1  # one invalid
    with L.Scheduler(p, alpha=(3, 2), method=method) as s:
        d, _ = s.schedule(sub)
        dag, opl, st = dev(sub.dag), dev(sub.op_local), dev(sub.start_us)
        obj = torch.empty(sub.n * p.n_hw, dtype=torch.int64, device="cuda")
        L.llama_backend_objectives(s.ctx, dag, opl, st, sub.now_us, obj)
        order = torch.empty(sub.n, dtype=torch.int32, device="cuda")
        aff = torch.empty(sub.n, dtype=torch.float64, device="cuda")
        L.llama_commit_order(s.ctx, dag, opl, dev(d.view(np.uint8)), obj, order, aff)
        got_obj = obj.cpu().numpy().reshape(sub.n, p.n_hw)
        got_order, got_aff = order.cpu().numpy(), aff.cpu().numpy()
    exp_obj = oracle.backend_objectives(p, sub, alpha=(3, 2))
    assert np.array_equal(got_obj, exp_obj)
    exp_order, exp_aff = oracle.commit_order(p, sub, d, exp_obj)
    assert np.array_equal(got_aff, exp_aff)
    assert np.array_equal(got_order, exp_order)


def test_queue_time_saturates_exactly_at_extreme_sums(L):
    """Eq. 2 (Section 4.3) with latencies near 2^31 and resources of 65,535: the
    exact per-backend sum exceeds 2^64 after about 1.3e5 such decisions.  The
    oracle sums exact integers and clamps the floored quotient to INT32_MAX;
    the device must give the same clamp (not a wrapped sum), and stay exact on
    a backend whose sum is small."""
    import torch
    p, inv = W.medium()
    p = copy.deepcopy(p)
    p.res = np.full(p.n_cfg, 65535, np.int32)
    p.res_total = np.asarray([1, 2**31 - 1, 1000], np.int32)
    n = 300_000
    idx = np.arange(n) % inv.n
    q_inv = inv.subset(idx)
    gop = p.dag_op_off[q_inv.dag] + q_inv.op_local
    hw = p.hw_off.reshape(p.n_ops, p.n_hw + 1)
    # backend of each decision: 0 and 1 alternate with extreme latencies, the
    # last 1,000 go to backend 2 with small ones
    lam = np.where(np.arange(n) % 2 == 0, 0, 1)
    lam[-1000:] = 2
    dec = np.zeros(n, dtype=L.DECISION_DTYPE)
    seg_start, seg_end = hw[gop, lam], hw[gop, lam + 1]
    has = seg_end > seg_start
    dec["cfg"] = np.where(has, seg_start, 0)
    dec["lat"] = np.where(lam == 2, 1000, 2**31 - 2)
    dec["flags"] = L.FLAG_FEASIBLE
    dec["cfg"][~has] = -1  # a backend with no configuration of that op: not queued
    with L.Scheduler(p) as s:
        q = torch.zeros(p.n_hw, dtype=torch.int64, device="cuda")
        L.llama_queue_time(s.ctx, dev(q_inv.dag), dev(q_inv.op_local), dev(dec.view(np.uint8)), q, apply=False)
        got = q.cpu().numpy()
    exp = oracle.queue_time(p, q_inv, dec)
    assert exp[0] == exp[1] == 2**31 - 1 and 0 < exp[2] < 2**31 - 1
    assert np.array_equal(got, exp), (got, exp)
