"""Hand-built problems for the tests: golden fixtures and closed-form shapes."""
import json
import os

import numpy as np

from paper_2102_01887_b300.workloads import Invocations, Problem

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name: str):
    with open(os.path.join(GOLDEN, name)) as f:
        g = json.load(f)
    pr = g["problem"]
    i32 = lambda k: np.asarray(pr[k], dtype=np.int32)
    i64 = lambda k: np.asarray(pr[k], dtype=np.int64)
    p = Problem(n_hw=pr["n_hw"], dag_op_off=i32("dag_op_off"), row_ptr=i32("row_ptr"),
                col=i32("col"), slo_us=i64("slo_us"), cfg_off=i64("cfg_off"), hw_off=i32("hw_off"),
                lat_us=i32("lat_us"), cost_nd=i64("cost_nd"), ref_cfg=i32("ref_cfg"),
                batch=i32("batch"), res=i32("res"), res_total=i32("res_total"), q_us=i64("q_us"))
    iv = g["invocations"]
    inv = Invocations(np.asarray(iv["dag"], np.int32), np.asarray(iv["op_local"], np.int32),
                      np.asarray(iv["start_us"], np.int64), int(iv["now_us"]))
    return g, p, inv


def single_table_problem(succ: list[list[int]], ref_lat: list[int], slo: int, q=(0, 0, 0),
                         extra: list[list[tuple[int, int, int]]] | None = None) -> Problem:
    """One DAG with local successor lists; op v gets its reference config (lat = ref_lat[v],
    on backend 0) plus optional extra configs (hw, lat, cost)."""
    n = len(succ)
    row_ptr, col = [0], []
    for s in succ:
        col.extend(s)
        row_ptr.append(len(col))
    lat, cost, hw_off, cfg_off = [], [], [], [0]
    for v in range(n):
        cfgs = [(0, ref_lat[v], ref_lat[v])] + list((extra or [[]] * n)[v])
        cfgs.sort(key=lambda c: c[0])
        ref_idx = cfgs.index((0, ref_lat[v], ref_lat[v]))
        lat += [c[1] for c in cfgs]
        cost += [c[2] for c in cfgs]
        hws = [c[0] for c in cfgs]
        hw_off += [int(np.searchsorted(hws, h, side="left")) for h in range(4)]
        cfg_off.append(cfg_off[-1] + len(cfgs))
        assert ref_idx == 0
    m = len(lat)
    return Problem(n_hw=3, dag_op_off=np.asarray([0, n], np.int32),
                   row_ptr=np.asarray(row_ptr, np.int32), col=np.asarray(col, np.int32),
                   slo_us=np.asarray([slo], np.int64), cfg_off=np.asarray(cfg_off, np.int64),
                   hw_off=np.asarray(hw_off, np.int32), lat_us=np.asarray(lat, np.int32),
                   cost_nd=np.asarray(cost, np.int64), ref_cfg=np.zeros(n, np.int32),
                   batch=np.ones(m, np.int32), res=np.ones(m, np.int32),
                   res_total=np.ones(3, np.int32), q_us=np.asarray(q, np.int64))


def staircase_select(p: Problem, v: int, slack_hw, mode: str = "cost_first", alpha=(1, 1)):
    """Independent selector: per backend, sort configurations by (L, index); the
    feasible ones for slack s are the prefix with L < s (binary search); keep a
    prefix-argmin of (cost, index) and, for alpha mode, a suffix-argmin of the
    infeasible objective; combine across backends.  Returns the op-local index."""
    first = int(p.cfg_off[v])
    hw = p.hw_off[v * (p.n_hw + 1):(v + 1) * (p.n_hw + 1)]
    cands = []
    for h in range(p.n_hw):
        xs = np.arange(hw[h], hw[h + 1])
        if xs.size == 0:
            continue
        L = p.lat_us[first + xs].astype(np.int64)
        C = p.cost_nd[first + xs].astype(np.int64)
        order = np.lexsort((xs, L))
        Ls, Cs, Xs = L[order], C[order], xs[order]
        k = int(np.searchsorted(Ls, int(slack_hw[h]), side="left"))  # number with L < s
        if k > 0:
            j = min(range(k), key=lambda t: (int(Cs[t]), int(Xs[t])))
            cands.append(((0, int(Cs[j]), int(Xs[j])) if mode == "cost_first"
                          else (int(Cs[j]), int(Xs[j]))))
        if mode == "alpha" and k < xs.size:
            objs = []
            for t in range(k, xs.size):
                g = first + int(Xs[t])
                term = (alpha[0] * int(p.lat_us[g]) * int(p.res[g])) // (
                    alpha[1] * int(p.batch[g]) * int(p.res_total[h]))
                objs.append((min(int(p.cost_nd[g]) + term, 2**63 - 1), int(Xs[t])))
            cands.append(min(objs))
    if mode == "alpha":
        return min(cands)[1]
    if cands:
        return min(cands)[2]
    n = int(p.cfg_off[v + 1]) - first
    return min(range(n), key=lambda x: (int(p.lat_us[first + x]), x))


def nx_source_sink_paths(p: Problem, d: int):
    """Every source-to-sink path of DAG d, enumerated by networkx."""
    import networkx as nx
    lo, hi = int(p.dag_op_off[d]), int(p.dag_op_off[d + 1])
    G = nx.DiGraph()
    G.add_nodes_from(range(lo, hi))
    for v in range(lo, hi):
        for e in range(p.row_ptr[v], p.row_ptr[v + 1]):
            G.add_edge(v, int(p.col[e]))
    sources = [v for v in G if G.in_degree(v) == 0]
    sinks = [v for v in G if G.out_degree(v) == 0]
    paths = []
    for s in sources:
        for t in sinks:
            paths.extend([[s]] if s == t else nx.all_simple_paths(G, s, t))
    return G, paths


def nx_invocation_slacks(p: Problem, inv: Invocations) -> np.ndarray:
    """Algorithm 1 over networkx-enumerated paths, with Python integers."""
    ref = p.lat_us[p.cfg_off[:-1] + p.ref_cfg].astype(np.int64)
    paths_of = {d: nx_source_sink_paths(p, d)[1] for d in set(int(x) for x in inv.dag)}
    out = np.zeros((inv.n, p.n_hw), dtype=np.int64)
    for i in range(inv.n):
        d = int(inv.dag[i])
        v = int(p.dag_op_off[d] + inv.op_local[i])
        rems = [sum(int(ref[u]) for u in path[path.index(v):]) for path in paths_of[d] if v in path]
        for h in range(p.n_hw):
            R = int(p.slo_us[d]) - (int(inv.now_us) - int(inv.start_us[i])) - int(p.q_us[h])
            out[i, h] = 0 if R <= 0 else min(int(ref[v]) * R // r for r in rems)
    return out
