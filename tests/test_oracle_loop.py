"""Pins of the serving-loop oracle (oracle/loop.py): a scenario worked out by
hand, and invariants on a larger random run.

The hand scenario: one DAG of one op, SLO 1,000 us, two backends; x0 on
backend 0 (L = 100 us, C/B = 10, R = 1) and x1 on backend 1 (L = 50, C/B =
30, R = 2), R_total = (1, 2); the reference configuration is x0, so the
critical path is 100 and slack(l) = 1000 - elapsed - Q[l] (Algorithm 1);
commit queues hold one invocation each.

tick 0: ten requests A..J (elapsed 0).  Q = (0, 0): both configurations are
  feasible, x0 is cheaper (Eq. 1), all ten go to SQ[0]; S_SQ[0] = 10 * 100.
  Late commit revisits A under Q = (1000 / 1, 0) = (1000, 0) (Eq. 2 counts the
  speculative queue): slack(0) = 0 makes x0 infeasible, x1 is feasible
  (50 < 1000) -> A commits into CQ[1] (slack 1000).
tick 1: Q = (900, 100 / 2 = 50); B's x0 has slack 100, not below it, so B
  would move to backend 1, whose commit queue is full: B stays.
tick 2: backend 1 dispatched A: Q = (900, 0), B commits into CQ[1] (slack 1000).
tick 3: backend 1 dispatched B; request K names a DAG that does not exist
  (rejected).  Q = (800, 0): C's x0 has slack 200 > 100, feasible and
  cheapest -> C commits into CQ[0] (slack 200).
"""
import numpy as np
import pytest

import oracle
from oracle.loop import COMMITTED, REJECTED, SPECULATED, LoopOracle
from paper_2102_01887_b300 import workloads as W


def micro_problem():
    return W.Problem(
        n_hw=2, dag_op_off=np.asarray([0, 1], np.int32), row_ptr=np.asarray([0, 0], np.int32),
        col=np.zeros(0, np.int32), slo_us=np.asarray([1000], np.int64), cfg_off=np.asarray([0, 2], np.int64),
        hw_off=np.asarray([0, 1, 2], np.int32), lat_us=np.asarray([100, 50], np.int32),
        cost_nd=np.asarray([10, 30], np.int64), ref_cfg=np.asarray([0], np.int32),
        batch=np.asarray([1, 1], np.int32), res=np.asarray([1, 2], np.int32),
        res_total=np.asarray([1, 2], np.int32), q_us=np.zeros(2, np.int64))


HAND_TICKS = [  # (submitted before the tick, now, dispatch, records)
    ([(i, 0, 0, 0) for i in range(10)], 0, (0, 0),
     [(i, SPECULATED, 0, 0, 100, 10, 1000, 1, 0) for i in range(10)]
     + [(0, COMMITTED, 0, 1, 50, 30, 1000, 1, 1)]),
    ([], 0, (0, 0), []),
    ([], 0, (0, 1), [(1, COMMITTED, 2, 1, 50, 30, 1000, 1, 1)]),
    ([(10, 5, 0, 0)], 0, (0, 1),
     [(10, REJECTED, 3, -1, 0, 0, 0, oracle.FLAG_INVALID, -1), (2, COMMITTED, 3, 0, 100, 10, 200, 1, 0)]),
]
HAND_QUEUES = [  # (Q after the tick, SQ lengths, CQ lengths)
    ((900, 50), (9, 0), (0, 1)), ((900, 50), (9, 0), (0, 1)), ((800, 50), (8, 0), (0, 1)),
    ((700 + 100, 0), (7, 0), (1, 0)),
]


def test_hand_scenario():
    lo = LoopOracle(micro_problem(), slots=10, max_admit=16, cq_cap=(1, 1))
    for (reqs, now, disp, want), (q, sq, cq) in zip(HAND_TICKS, HAND_QUEUES):
        lo.submit(reqs)
        assert lo.tick(now, disp) == want
        assert lo.queueing_time().tolist() == list(q)
        assert [len(x) for x in lo.sq] == list(sq) and [len(x) for x in lo.cq] == list(cq)


def test_slots_bound_admission():
    lo = LoopOracle(micro_problem(), slots=3, max_admit=16, cq_cap=(1, 1))
    lo.submit([(i, 0, 0, 0) for i in range(5)])
    out = lo.tick(0, (0, 0))
    assert [r[0] for r in out if r[1] == SPECULATED] == [0, 1, 2]  # three slots
    assert len(lo.pending) == 2
    out = lo.tick(0, (0, 0))  # nothing dispatched: no slot frees, nothing admitted
    assert not [r for r in out if r[1] == SPECULATED]
    # A was committed to backend 0 (Q = (300, 0) leaves x0 feasible): backend 0
    # dispatching it frees a slot, and the next request is admitted
    out = lo.tick(0, (1, 0))
    assert [r[0] for r in out if r[1] == SPECULATED] == [3]


def run_random(p, seed, ticks=12, mode=0, alpha=(1, 1), slots=4000, cq=(40, 24, 16)):
    rng = np.random.default_rng(seed)
    _, inv = W.medium(n_inv=4000, inv_seed=seed)
    lo = LoopOracle(p, slots=slots, max_admit=1024, cq_cap=cq, mode=mode, alpha=alpha)
    now, k, recs = int(inv.now_us) - 200_000, 0, []
    for t in range(ticks):
        n = int(rng.integers(0, 500))
        batch = [(k + j, int(inv.dag[k + j]), int(inv.op_local[k + j]), int(inv.start_us[k + j]) - 300_000)
                 for j in range(min(n, inv.n - k))]
        k += len(batch)
        lo.submit(batch)
        recs += lo.tick(now, rng.integers(0, 30, p.n_hw))
        now += int(rng.integers(0, 40_000))
    return lo, recs


def test_random_run_invariants():
    p, _ = W.medium()
    lo, recs = run_random(p, 3)
    spec = [r for r in recs if r[1] == SPECULATED]
    com = [r for r in recs if r[1] == COMMITTED]
    assert len({r[0] for r in spec}) == len(spec) and len({r[0] for r in com}) == len(com)
    assert {r[0] for r in com} <= {r[0] for r in spec}  # only admitted invocations commit
    assert com and len(com) < len(spec)
    # the queues' contents give the queueing time (Eq. 2 over both queues)
    hw = p.hw_off.reshape(p.n_ops, p.n_hw + 1)
    for h in range(p.n_hw):
        assert sum(e["lr"] for e in lo.sq[h]) == lo.s_sq[h]
        assert sum(e["lr"] for e in lo.cq[h]) == lo.s_cq[h]
        assert len(lo.cq[h]) <= lo.cq_cap[h]
    # a committed configuration belongs to the commit queue's backend
    for r in com:
        assert r[8] in range(p.n_hw)
    del hw


def two_op_problem():
    """Two DAGs of one op each, SLO 10,000 us: u with x0 (backend 0: L 100, C/B 10,
    R 1) and x1 (backend 1: L 50, C/B 30, R 2); w with y0 (backend 0: L 300,
    C/B 5, R 1) and y1 (backend 1: L 200, C/B 40, R 2); R_total = (1, 2)."""
    return W.Problem(
        n_hw=2, dag_op_off=np.asarray([0, 1, 2], np.int32), row_ptr=np.asarray([0, 0, 0], np.int32),
        col=np.zeros(0, np.int32), slo_us=np.asarray([10_000, 10_000], np.int64),
        cfg_off=np.asarray([0, 2, 4], np.int64), hw_off=np.asarray([0, 1, 2, 0, 1, 2], np.int32),
        lat_us=np.asarray([100, 50, 300, 200], np.int32), cost_nd=np.asarray([10, 30, 5, 40], np.int64),
        ref_cfg=np.asarray([0, 0], np.int32), batch=np.ones(4, np.int32), res=np.asarray([1, 2, 1, 2], np.int32),
        res_total=np.asarray([1, 2], np.int32), q_us=np.zeros(2, np.int64))


# Two ops, commit queues of two: U1 (u) and W1 (w) both speculate onto backend 0
# (Q = 0; the cheapest feasible configurations x0 and y0).  Revisited under
# Q = (100 + 300, 0) both stay on backend 0 (slack 9,600); W1 commits first:
# its affinity is 40 / 5 = 8 (least objective on backend 1 over backend 0's),
# U1's 30 / 10 = 3.  Tick 1: backend 0 dispatched its head, W1 (L R = 300), so
# U2 speculates under Q = (100, 0) (slack 9,900) and commits under (200, 0).
TWO_OP_TICKS = [
    ([(100, 0, 0, 0), (101, 1, 0, 0)], 0, (0, 0),
     [(100, SPECULATED, 0, 0, 100, 10, 10_000, 1, 0), (101, SPECULATED, 0, 0, 300, 5, 10_000, 1, 0),
      (101, COMMITTED, 0, 0, 300, 5, 9_600, 1, 0), (100, COMMITTED, 0, 0, 100, 10, 9_600, 1, 0)]),
    ([(102, 0, 0, 0)], 0, (1, 0),
     [(102, SPECULATED, 1, 0, 100, 10, 9_900, 1, 0), (102, COMMITTED, 1, 0, 100, 10, 9_800, 1, 0)]),
]


def pin_loop(mod) -> list[str]:
    """Hand-worked scenarios against a (possibly mutated) oracle module."""
    failed = []
    lo = mod.LoopOracle(micro_problem(), slots=10, max_admit=16, cq_cap=(1, 1))
    for t, ((reqs, now, disp, want), (q, sq, cq)) in enumerate(zip(HAND_TICKS, HAND_QUEUES)):
        lo.submit(reqs)
        if lo.tick(now, disp) != want or lo.queueing_time().tolist() != list(q):
            failed.append(f"hand_tick_{t}")
            break
    # three slots: requests 0, 1, 2 speculate (Q = 0), A = 0 commits into CQ[0]
    # (Q = (300, 0), slack 700); after backend 0 dispatches it, request 3
    # speculates under Q = (200, 0) and B commits under (300, 0)
    lo = mod.LoopOracle(micro_problem(), slots=3, max_admit=16, cq_cap=(1, 1))
    lo.submit([(i, 0, 0, 0) for i in range(5)])
    firsts = [r[0] for r in lo.tick(0, (0, 0)) if r[1] == SPECULATED]
    lo.tick(0, (0, 0))
    if firsts != [0, 1, 2] or lo.tick(0, (1, 0)) != [(3, SPECULATED, 2, 0, 100, 10, 800, 1, 0),
                                                     (1, COMMITTED, 2, 0, 100, 10, 700, 1, 0)]:
        failed.append("slots")
    lo = mod.LoopOracle(two_op_problem(), slots=10, max_admit=16, cq_cap=(2, 2))
    for t, (reqs, now, disp, want) in enumerate(TWO_OP_TICKS):
        lo.submit(reqs)
        if lo.tick(now, disp) != want:
            failed.append(f"two_op_tick_{t}")
            break
    # one place in CQ[0]: the head of SQ[0], U1, is the only candidate
    lo = mod.LoopOracle(two_op_problem(), slots=10, max_admit=16, cq_cap=(1, 2))
    lo.submit(TWO_OP_TICKS[0][0])
    if [r[0] for r in lo.tick(0, (0, 0)) if r[1] == COMMITTED] != [100]:
        failed.append("fifo_head")
    # a rejected request takes no slot: with two slots, 201 and then 202 are admitted
    lo = mod.LoopOracle(micro_problem(), slots=2, max_admit=16, cq_cap=(1, 1))
    lo.submit([(200, 5, 0, 0), (201, 0, 0, 0), (202, 0, 0, 0)])
    lo.tick(0, (0, 0))
    if lo.tick(0, (0, 0)) != [(202, SPECULATED, 1, 0, 100, 10, 900, 1, 0)]:
        failed.append("rejected_slot")
    return failed


LOOP_MUTANTS = {
    "commit_sees_commit_queue_only": ("        q1 = self.queueing_time()\n",
                                      "        q1 = np.asarray([min(self.s_cq[h] // int(self.p.res_total[h]), "
                                      "INT32_MAX) for h in range(self.H)], np.int64)\n"),
    "speculation_ignores_queues": ("        q0 = self.queueing_time()\n", "        q0 = np.zeros(self.H, np.int64)\n"),
    "commit_to_source_backend": ("                if room[lam] <= 0:", "                lam = h_src\n                if room[lam] <= 0:"),
    "no_commit_capacity": ("                if room[lam] <= 0:\n                    continue", "                pass"),
    "lifo_speculative_queue": ("self.sq[lam].append(e)", "self.sq[lam].appendleft(e)"),
    "dispatch_from_tail": ("e = self.cq[h].popleft()", "e = self.cq[h].pop()"),
    "rejected_take_slots": ("                if d[\"flags\"] & FLAG_INVALID:\n",
                            "                if d[\"flags\"] & FLAG_INVALID:\n                    self.free -= 1\n"),
}


def test_loop_oracle_passes_its_pins():
    import oracle.loop as real
    assert pin_loop(real) == []


@pytest.mark.parametrize("name", sorted(LOOP_MUTANTS))
def test_loop_mutant_is_caught(name, tmp_path):
    import importlib.util
    import os
    old, new = LOOP_MUTANTS[name]
    src = open(os.path.join(os.path.dirname(oracle.__file__), "loop.py")).read()
    assert src.count(old) == 1, f"mutation site not unique: {old!r}"
    path = tmp_path / "loop_mutant.py"
    path.write_text(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("oracle.loop_mutant", path)
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = "oracle"
    spec.loader.exec_module(mod)
    assert pin_loop(mod), f"mutant {name} passed every pin"
