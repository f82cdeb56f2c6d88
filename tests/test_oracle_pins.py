"""Pins of the CPU oracle to things other than itself.

* a hand-derived worked example (tests/golden/amber_worked_example.json);
* networkx path enumeration for Algorithm 1 (Section 4.1) and the longest
  remaining path;
* closed forms: a chain, a single operation, a sink, the AMBER Alert shape;
* an independent selector (sort by latency + binary search + prefix argmin)
  for the cost-first reading of Eq. 1 (Section 4.2) and for alpha mode;
* invariants of the method, and special cases of alpha mode that reduce to
  plain argmins.
"""
import numpy as np
import networkx as nx
import pytest

import oracle
from paper_2102_01887_b300 import workloads as W
from tests.problems import load_golden, single_table_problem, staircase_select


# ---------------------------------------------------------------- golden ---

def test_golden_critical_path_and_slack():
    g, p, inv = load_golden("amber_worked_example.json")
    assert oracle.critical_path(p).tolist() == g["expected_critical_path"]
    for method in ("critical_path", "paths"):
        assert oracle.slacks(p, inv, method).tolist() == g["expected_slack"]


@pytest.mark.parametrize("mode", ["cost_first", "alpha"])
def test_golden_decisions(mode):
    g, p, inv = load_golden("amber_worked_example.json")
    m = oracle.MODE_COST_FIRST if mode == "cost_first" else oracle.MODE_ALPHA
    for method in ("critical_path", "paths"):
        d, rc = oracle.schedule(p, inv, mode=m, alpha=tuple(g["alpha"]), method=method)
        assert rc == oracle.OK
        exp = g["expected_" + mode]
        for k in ("cfg", "lat", "cost", "slack", "flags"):
            assert d[k].tolist() == exp[k], (mode, method, k)


# ------------------------------------------------- networkx enumeration ---

def _graph(p, d):
    lo, hi = int(p.dag_op_off[d]), int(p.dag_op_off[d + 1])
    G = nx.DiGraph()
    G.add_nodes_from(range(lo, hi))
    for v in range(lo, hi):
        for e in range(p.row_ptr[v], p.row_ptr[v + 1]):
            G.add_edge(v, int(p.col[e]))
    return G


def _nx_paths(G):
    sources = [v for v in G if G.in_degree(v) == 0]
    sinks = [v for v in G if G.out_degree(v) == 0]
    paths = []
    for s in sources:
        for t in sinks:
            if s == t:
                paths.append([s])
            else:
                paths.extend(nx.all_simple_paths(G, s, t))
    return paths


@pytest.mark.parametrize("seed", range(40))
def test_slack_matches_networkx_path_enumeration(seed):
    p, inv = W.random_small(seed)
    ref = oracle.reference_latency(p)
    cp = oracle.critical_path(p)
    for d in range(p.n_dags):
        G = _graph(p, d)
        paths = _nx_paths(G)
        for v in G:
            # longest remaining path from v, v included
            rem = [sum(int(ref[u]) for u in path[path.index(v):]) for path in paths if v in path]
            assert rem, "every op lies on a source-to-sink path"
            assert cp[v] == max(rem)
            for R in (-5, 0, 1, 7, 123, 10**6 + 3):
                expect = 0 if R <= 0 else min(int(ref[v]) * R // r for r in rem)
                got, n_paths = oracle.slack_paths(p, v, R)
                assert got == expect
                assert n_paths == len(paths)
                assert oracle.load().or_slack_from_cp(int(ref[v]), int(cp[v]), R) == expect


# --------------------------------------------------------- closed forms ---

def test_chain_closed_form():
    ref = [70, 10, 30, 5, 45]
    p = single_table_problem([[1], [2], [3], [4], []], ref, slo=1000)
    for v in range(5):
        for R in (1, 99, 1000, 123457):
            exp = ref[v] * R // sum(ref[v:])
            assert oracle.slack_paths(p, v, R)[0] == exp
            assert oracle.load().or_slack_from_cp(ref[v], sum(ref[v:]), R) == exp
    assert oracle.critical_path(p).tolist() == [sum(ref[v:]) for v in range(5)]


def test_single_op_and_sink_get_all_remaining_time():
    p = single_table_problem([[]], [37], slo=500)
    for R in (1, 36, 37, 10**9):
        assert oracle.slack_paths(p, 0, R)[0] == R
    p = single_table_problem([[1, 2], [], []], [10, 20, 30], slo=500)
    for v in (1, 2):
        assert oracle.slack_paths(p, v, 777)[0] == 777


def test_amber_shape_closed_form():
    # decode -> detect -> {face | car}: detect's slack uses the longer branch
    ref = [100, 400, 300, 200]
    p = single_table_problem([[1], [2, 3], [], []], ref, slo=2000)
    for R in (1, 700, 1400, 99991):
        assert oracle.slack_paths(p, 1, R)[0] == 400 * R // (400 + max(300, 200))
        assert oracle.slack_paths(p, 0, R)[0] == 100 * R // (100 + 400 + 300)


def test_passed_target_gives_zero_slack_and_fastest_config():
    p = single_table_problem([[]], [50], slo=100, extra=[[(1, 20, 900), (2, 10, 999), (2, 10, 5)]])
    inv = W.Invocations(np.zeros(3, np.int32), np.zeros(3, np.int32),
                        np.asarray([0, 0, 50], np.int64), 150)  # elapsed 150, 150, 100
    d, rc = oracle.schedule(p, inv)
    assert rc == oracle.OK
    assert d["slack"].tolist() == [0, 0, 0]
    assert d["cfg"].tolist() == [2, 2, 2]  # L=10 twice: lowest index wins
    assert d["flags"].tolist() == [0, 0, 0]


# ------------------------------------------------- independent selector ---

@pytest.mark.parametrize("seed", range(60))
@pytest.mark.parametrize("mode", ["cost_first", "alpha"])
def test_selection_matches_staircase(seed, mode):
    p, inv = W.random_small(seed)
    alpha = (int(1 + seed % 5), int(1 + (seed * 7) % 3))
    d, rc = oracle.schedule(p, inv, mode=oracle.MODE_ALPHA if mode == "alpha" else 0, alpha=alpha)
    assert rc == oracle.OK
    sl = oracle.slacks(p, inv)
    for i in range(inv.n):
        v = int(p.dag_op_off[inv.dag[i]] + inv.op_local[i])
        assert d["cfg"][i] == staircase_select(p, v, sl[i], mode, alpha)


def test_selection_matches_staircase_medium_sample():
    p, inv = W.medium()
    sub = inv.subset(np.arange(0, inv.n, 257))
    d, rc = oracle.schedule(p, sub)
    assert rc == oracle.OK
    sl = oracle.slacks(p, sub)
    for i in range(sub.n):
        v = int(p.dag_op_off[sub.dag[i]] + sub.op_local[i])
        assert d["cfg"][i] == staircase_select(p, v, sl[i])


# ------------------------------------------------------------ invariants ---

def _check_invariants(p, inv, d, sl):
    for i in range(inv.n):
        v = int(p.dag_op_off[inv.dag[i]] + inv.op_local[i])
        lo, hi = int(p.cfg_off[v]), int(p.cfg_off[v + 1])
        hw = p.hw_off[v * (p.n_hw + 1):(v + 1) * (p.n_hw + 1)]
        lam = np.searchsorted(hw, np.arange(hi - lo), side="right") - 1
        L = p.lat_us[lo:hi].astype(np.int64)
        C = p.cost_nd[lo:hi]
        feas = L < sl[i][lam]
        x = int(d["cfg"][i])
        assert d["lat"][i] == L[x] and d["cost"][i] == C[x] and d["slack"][i] == sl[i][lam[x]]
        assert bool(d["flags"][i] & oracle.FLAG_FEASIBLE) == bool(feas[x])
        assert feas[x] == feas.any()  # feasible whenever any config is
        if feas.any():
            assert C[x] == C[feas].min()  # cheapest feasible
            assert x == np.flatnonzero(feas & (C == C[x]))[0]  # lowest index among ties
        else:
            assert L[x] == L.min()  # otherwise the fastest
            assert x == np.flatnonzero(L == L[x])[0]


@pytest.mark.parametrize("seed", range(30))
def test_selection_invariants(seed):
    p, inv = W.random_small(seed + 1000, max_cfg=12)
    d, rc = oracle.schedule(p, inv)
    assert rc == oracle.OK
    sl = oracle.slacks(p, inv)
    # slack never exceeds the remaining time, never negative
    t = inv.now_us - inv.start_us
    R = p.slo_us[inv.dag][:, None] - t[:, None] - p.q_us[None, :]
    assert (sl >= 0).all() and (sl <= np.maximum(R, 0)).all()
    _check_invariants(p, inv, d, sl)


def test_slack_monotone_in_elapsed_time_and_queueing():
    p, inv = W.medium()
    sub = inv.subset(np.arange(0, inv.n, 97))
    s0 = oracle.slacks(p, sub)
    later = W.Invocations(sub.dag, sub.op_local, sub.start_us - 12_345, sub.now_us)
    assert (oracle.slacks(p, later) <= s0).all()
    p.q_us = p.q_us + np.asarray([0, 5_000, 50_000])
    s2 = oracle.slacks(p, sub)
    assert (s2 <= s0).all() and (s2[:, 0] == s0[:, 0]).all()


def test_misprofiling_halved_latencies_only_enlarge_feasible_set():
    # Section 6.4 mis-profiling experiment: every profiled latency set to 50%.
    # Start from a table of even latencies so that halving is exact; then the
    # reference latencies and the critical path halve exactly, the slack is
    # unchanged, and the feasible set can only grow.
    p, inv = W.medium()
    sub = inv.subset(np.arange(0, inv.n, 131))
    true = W.Problem(**{**p.__dict__, "lat_us": (p.lat_us * 2).astype(np.int32)})
    d0, _ = oracle.schedule(true, sub)
    d1, _ = oracle.schedule(p, sub)
    sl0, sl1 = oracle.slacks(true, sub), oracle.slacks(p, sub)
    assert (sl0 == sl1).all()
    for i in range(sub.n):
        v = int(p.dag_op_off[sub.dag[i]] + sub.op_local[i])
        lo, hi = int(p.cfg_off[v]), int(p.cfg_off[v + 1])
        hw = p.hw_off[v * 4:(v + 1) * 4]
        lam = np.searchsorted(hw, np.arange(hi - lo), side="right") - 1
        f0 = true.lat_us[lo:hi] < sl0[i][lam]
        f1 = p.lat_us[lo:hi] < sl1[i][lam]
        assert (f1 | ~f0).all()
        if f0.any():  # the cheapest feasible config can only get cheaper
            assert d1["cost"][i] <= d0["cost"][i]
    assert (d1["flags"] & 1).sum() >= (d0["flags"] & 1).sum()


# ------------------------------------------------- alpha special cases ---

def test_alpha_negligible_weight_is_plain_cheapest():
    # alpha * L * R / (B * R_total) < 1 everywhere -> objective = C/B for all x
    p, inv = W.random_small(7, max_cfg=12)
    p.res_total = np.full(3, 10**6, np.int32)
    d, rc = oracle.schedule(p, inv, mode=oracle.MODE_ALPHA, alpha=(1, 65535))
    assert rc == oracle.OK
    for i in range(inv.n):
        v = int(p.dag_op_off[inv.dag[i]] + inv.op_local[i])
        lo, hi = int(p.cfg_off[v]), int(p.cfg_off[v + 1])
        C = p.cost_nd[lo:hi]
        assert d["cfg"][i] == int(np.flatnonzero(C == C.min())[0])


def test_alpha_dominant_weight_prefers_feasible_then_throughput():
    # B = R = R_total = 1 and alpha larger than any cost gap: any feasible config beats
    # any infeasible one, and among infeasible ones the order is (L, cost, index).
    p, inv = W.random_small(11, max_cfg=12)
    p.batch[:] = 1
    p.res[:] = 1
    p.res_total[:] = 1
    d, rc = oracle.schedule(p, inv, mode=oracle.MODE_ALPHA, alpha=(1000, 1))
    assert rc == oracle.OK
    sl = oracle.slacks(p, inv)
    for i in range(inv.n):
        v = int(p.dag_op_off[inv.dag[i]] + inv.op_local[i])
        lo, hi = int(p.cfg_off[v]), int(p.cfg_off[v + 1])
        hw = p.hw_off[v * 4:(v + 1) * 4]
        lam = np.searchsorted(hw, np.arange(hi - lo), side="right") - 1
        L, C = p.lat_us[lo:hi], p.cost_nd[lo:hi]
        feas = L < sl[i][lam]
        if feas.any():
            exp = min(np.flatnonzero(feas), key=lambda x: (C[x], x))
        else:
            exp = min(range(hi - lo), key=lambda x: (L[x], C[x], x))
        assert d["cfg"][i] == exp


# -------------------------------------------------------- invalid input ---

def test_invalid_invocations_flagged():
    g, p, inv = load_golden("amber_worked_example.json")
    bad = W.Invocations(np.asarray([0, 1, 0, 0, -1], np.int32), np.asarray([1, 0, 4, 2, 0], np.int32),
                        np.asarray([9400, 9400, 9400, 10001, 0], np.int64), 10000)
    d, rc = oracle.schedule(p, bad)
    assert rc == oracle.EINVAL
    assert d["cfg"].tolist() == [5, -1, -1, -1, -1]
    assert d["flags"].tolist() == [1, 2, 2, 2, 2]


def test_cycle_rejected():
    p = single_table_problem([[1], [0]], [1, 1], slo=10)
    with pytest.raises(ValueError):
        oracle.critical_path(p)
