"""Pins of the oracle's Eq. 2 (queueing time) on hand-built cases."""
import numpy as np

import oracle
from tests.problems import load_golden


def test_queue_time_hand_computed():
    g, p, inv = load_golden("amber_worked_example.json")
    p.res = np.arange(1, p.n_cfg + 1, dtype=np.int32) % 4 + 1
    p.res_total = np.asarray([3, 7, 5][:p.n_hw], np.int32)
    d, _ = oracle.schedule(p, inv)
    hw = p.hw_off.reshape(p.n_ops, p.n_hw + 1)
    want = [0] * p.n_hw
    for i in range(inv.n):
        if d["cfg"][i] < 0:
            continue
        v = p.dag_op_off[inv.dag[i]] + inv.op_local[i]
        x = int(d["cfg"][i])
        lam = int(np.searchsorted(hw[v], x, side="right")) - 1
        want[lam] += int(d["lat"][i]) * int(p.res[p.cfg_off[v] + x])
    want = [w // int(p.res_total[h]) for h, w in enumerate(want)]
    assert oracle.queue_time(p, inv, d).tolist() == want


def test_queue_time_skips_invalid_and_floors_once():
    # two decided invocations of op 1 on backend 1 with latency 3 and R = 1,
    # R_total = 2: Q = floor(6 / 2) = 3 (flooring each term would give 1 + 1);
    # a third, invalid, decision is skipped; the other backends are empty
    g, p, inv = load_golden("amber_worked_example.json")
    p.res = np.ones(p.n_cfg, np.int32)
    p.res_total = np.full(p.n_hw, 2, np.int32)
    hw = p.hw_off.reshape(p.n_ops, p.n_hw + 1)
    v = 1
    x = int(hw[v, 1])
    assert hw[v, 2] > x  # backend 1 of op 1 is not empty
    import paper_2102_01887_b300.workloads as W
    q_inv = W.Invocations(np.zeros(3, np.int32), np.full(3, v - p.dag_op_off[0], np.int32),
                          np.zeros(3, np.int64), 10)
    d = np.zeros(3, oracle.DECISION_DTYPE)
    d["cfg"] = [x, x, x]
    d["lat"] = [3, 3, 1000]
    d["flags"] = [0, 0, oracle.FLAG_INVALID]
    q = oracle.queue_time(p, q_inv, d)
    assert q.tolist() == [0, 3, 0][:p.n_hw]


def test_feedback_closed_forms():
    import copy
    g, p0, inv = load_golden("amber_worked_example.json")
    v, x = 1, 2
    gidx = int(p0.cfg_off[v]) + x
    # beta = 1: the observation replaces the table entry; beta = 0: nothing moves
    p = copy.deepcopy(p0)
    oracle.feedback(p, [v], [x], [777], [55], beta=(1, 1))
    assert p.lat_us[gidx] == 777 and p.cost_nd[gidx] == 55
    p = copy.deepcopy(p0)
    oracle.feedback(p, [v], [x], [777], [55], beta=(0, 5))
    assert np.array_equal(p.lat_us, p0.lat_us) and np.array_equal(p.cost_nd, p0.cost_nd)
    # beta = 1/2 from 100: 101 -> (100 + 101 + 1) // 2 = 101 (halves round up)
    p = copy.deepcopy(p0)
    p.lat_us[gidx] = 100
    oracle.feedback(p, [v], [x], [101], [0], beta=(1, 2))
    assert p.lat_us[gidx] == 101
    # order matters: from 100 with beta 1/2, 200 then 400 gives 150 then 275; 400 then 200
    # gives 250 then 225
    p = copy.deepcopy(p0)
    p.lat_us[gidx] = 100
    oracle.feedback(p, [v, v], [x, x], [200, 400], [0, 0], beta=(1, 2))
    assert p.lat_us[gidx] == 275
    p.lat_us[gidx] = 100
    oracle.feedback(p, [v, v], [x, x], [400, 200], [0, 0], beta=(1, 2))
    assert p.lat_us[gidx] == 225
    # observations outside the tables are skipped
    assert oracle.feedback(p, [-1, v, v], [0, 10**6, x], [5, 5, 0], [0, 0, 0]) == 3


def test_backend_minima_agree_with_the_alpha_decision():
    # the least of an invocation's per-backend minima is the objective of the
    # configuration Eq. 1 selects (the C oracle's alpha mode, another code path)
    from paper_2102_01887_b300 import workloads as W
    for seed in range(6):
        p, inv = W.random_small(seed, max_cfg=12, n_inv=40)
        a = (2 + seed % 3, 3)
        obj = oracle.backend_objectives(p, inv, alpha=a)
        d, _ = oracle.schedule(p, inv, mode=oracle.MODE_ALPHA, alpha=a)
        sl = oracle.slacks(p, inv)
        hw = p.hw_off.reshape(p.n_ops, p.n_hw + 1)
        for i in range(inv.n):
            if d["flags"][i] & oracle.FLAG_INVALID:
                assert (obj[i] == 2**63 - 1).all()
                continue
            v = p.dag_op_off[inv.dag[i]] + inv.op_local[i]
            x = int(d["cfg"][i])
            g = p.cfg_off[v] + x
            lam = int(np.searchsorted(hw[v], x, side="right")) - 1
            L, C = int(p.lat_us[g]), int(p.cost_nd[g])
            want = C if L < sl[i, lam] else C + (a[0] * L * int(p.res[g])) // (a[1] * int(p.batch[g]) * int(p.res_total[lam]))
            assert obj[i].min() == want, (seed, i)


def test_commit_order_invariants():
    from paper_2102_01887_b300 import workloads as W
    p, inv = W.random_small(3, max_cfg=10, n_inv=60)
    d, _ = oracle.schedule(p, inv)
    obj = oracle.backend_objectives(p, inv, alpha=(1, 1))
    order, aff = oracle.commit_order(p, inv, d, obj)
    assert sorted(order.tolist()) == list(range(inv.n))
    hw = p.hw_off.reshape(p.n_ops, p.n_hw + 1)
    lam = []
    for i in order:
        if d["cfg"][i] < 0:
            lam.append(p.n_hw)
        else:
            v = p.dag_op_off[inv.dag[i]] + inv.op_local[i]
            lam.append(int(np.searchsorted(hw[v], d["cfg"][i], side="right")) - 1)
    assert lam == sorted(lam)  # grouped by backend
    for k in range(1, inv.n):  # within a backend: affinity descending, then index
        if lam[k] == lam[k - 1] and lam[k] < p.n_hw:
            i, j = order[k - 1], order[k]
            assert aff[i] > aff[j] or (aff[i] == aff[j] and i < j)
