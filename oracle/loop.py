"""Plain sequential simulation of the serving loop with early speculation and
late commit (Section 4.3) and priority-based commit (Section 4.4) -- TEST
INFRASTRUCTURE, like the rest of ``oracle/``: only the tests and the
benchmark's CPU legs use it.

One tick, in the order of Section 4.3:

1. dispatch: each backend took ``dispatch[l]`` invocations from the head of
   its commit queue CQ[l]; they leave the queue and free their slots;
2. admit: pending requests, in arrival order, while slots are free, at most
   ``max_admit``; an invalid one is rejected (it takes no slot);
3. early speculation: every admitted invocation gets its slack (Algorithm 1)
   under the queueing time at the tick's start, Q[l] = floor(sum over SQ[l]
   and CQ[l] of L(x_i) R(x_i) / R_total(l)) (Eq. 2 over both queues, the exact
   sum floored once), and the configuration Eq. 1 selects; it joins the back
   of SQ[l(x)], in arrival order;
4. late commit: the first cq_cap[l] entries of every SQ[l] are revisited --
   Algorithm 1 and Eq. 1 again under the queueing time after step 3 (both
   queues, the candidates themselves included) -- and committed into the
   commit queue of their new backend l' in the order of Section 4.4 (by l',
   then descending Eq. 3 affinity, then candidate order), while CQ[l'] has
   room; the others stay in their SQ with their speculative decision.

Decisions are the C oracle's (``oracle.schedule``); the Eq. 3 affinities and
order are ``oracle.backend_objectives`` and ``oracle.commit_order``.
"""
from __future__ import annotations

import copy
from collections import deque

import numpy as np

from . import FLAG_INVALID, MODE_COST_FIRST, schedule, backend_objectives, commit_order

INT32_MAX = 2**31 - 1
SPECULATED, COMMITTED, REJECTED = 1, 2, 3


class LoopOracle:
    def __init__(self, p, slots: int, max_admit: int, cq_cap, mode: int = MODE_COST_FIRST, alpha=(1, 1)):
        self.p = copy.deepcopy(p)
        self.H = p.n_hw
        self.mode, self.alpha = mode, tuple(alpha)
        self.free = int(slots)
        self.max_admit = int(max_admit)
        self.cq_cap = [int(c) for c in cq_cap[:self.H]]
        self.sq = [deque() for _ in range(self.H)]
        self.cq = [deque() for _ in range(self.H)]
        self.s_sq = [0] * self.H  # exact sums of L(x) R(x) over each queue
        self.s_cq = [0] * self.H
        self.pending = deque()
        self.ticks = 0
        self.q_log = []  # per tick: (queueing time at speculation, at commit)
        self.hw = p.hw_off.reshape(p.n_ops, self.H + 1)

    def submit(self, reqs):
        """reqs: iterable of (id, dag, op_local, start_us)."""
        for r in reqs:
            self.pending.append(tuple(int(v) for v in r))

    def queueing_time(self) -> np.ndarray:
        """Eq. 2 over both queues of every backend."""
        rt = self.p.res_total
        return np.asarray([min((self.s_sq[h] + self.s_cq[h]) // int(rt[h]), INT32_MAX) for h in range(self.H)],
                          np.int64)

    def _op(self, dag: int, opl: int) -> int:
        return int(self.p.dag_op_off[dag]) + opl

    def _backend(self, v: int, x: int) -> int:
        return max(h for h in range(self.H) if x >= self.hw[v, h])

    def _lr(self, v: int, dec) -> int:
        return int(dec["lat"]) * int(self.p.res[int(self.p.cfg_off[v]) + int(dec["cfg"])])

    def _decide(self, entries, now: int, q):
        """Decisions of Eq. 1 for (dag, op_local, start) entries under queueing time q."""
        from paper_2102_01887_b300.workloads import Invocations
        inv = Invocations(np.asarray([e[0] for e in entries], np.int32),
                          np.asarray([e[1] for e in entries], np.int32),
                          np.asarray([e[2] for e in entries], np.int64), int(now))
        self.p.q_us = np.asarray(q, np.int64)
        dec, _ = schedule(self.p, inv, mode=self.mode, alpha=self.alpha)
        return inv, dec

    def tick(self, now: int, dispatch=None):
        """One tick; returns its records: (id, kind, tick, cfg, lat, cost, slack, flags, backend)."""
        out = []
        t = self.ticks
        # 1. dispatch
        for h in range(self.H):
            k = min(int(dispatch[h]) if dispatch is not None else 0, len(self.cq[h]))
            for _ in range(k):
                e = self.cq[h].popleft()
                self.s_cq[h] -= e["lr"]
                self.free += 1
        # 2. admit
        n = min(len(self.pending), self.free, self.max_admit)
        batch = [self.pending.popleft() for _ in range(n)]
        # 3. early speculation under the queueing time at the tick's start
        q0 = self.queueing_time()
        if batch:
            _, dec = self._decide([(b[1], b[2], b[3]) for b in batch], now, q0)
            for b, d in zip(batch, dec):
                if d["flags"] & FLAG_INVALID:
                    out.append((b[0], REJECTED, t, -1, 0, 0, 0, int(d["flags"]), -1))
                    continue
                v = self._op(b[1], b[2])
                lam = self._backend(v, int(d["cfg"]))
                e = {"id": b[0], "dag": b[1], "opl": b[2], "start": b[3], "lr": self._lr(v, d)}
                self.sq[lam].append(e)
                self.s_sq[lam] += e["lr"]
                self.free -= 1
                out.append((b[0], SPECULATED, t, int(d["cfg"]), int(d["lat"]), int(d["cost"]), int(d["slack"]),
                            int(d["flags"]), lam))
        # 4. late commit: the heads of every speculative queue, re-scored together
        cand = [(h, e) for h in range(self.H) for e in list(self.sq[h])[:self.cq_cap[h]]]
        q1 = self.queueing_time()
        self.q_log.append((q0, q1))
        if cand:
            inv, dec = self._decide([(e["dag"], e["opl"], e["start"]) for _, e in cand], now, q1)
            self.p.q_us = q1
            obj = backend_objectives(self.p, inv, alpha=self.alpha)
            order, _ = commit_order(self.p, inv, dec, obj)
            room = [self.cq_cap[h] - len(self.cq[h]) for h in range(self.H)]
            committed = set()
            for k in order:
                h_src, e = cand[k]
                d = dec[k]
                v = self._op(e["dag"], e["opl"])
                lam = self._backend(v, int(d["cfg"]))
                if room[lam] <= 0:
                    continue
                room[lam] -= 1
                committed.add(id(e))
                self.s_sq[h_src] -= e["lr"]
                ce = dict(e, lr=self._lr(v, d))
                self.cq[lam].append(ce)
                self.s_cq[lam] += ce["lr"]
                out.append((e["id"], COMMITTED, t, int(d["cfg"]), int(d["lat"]), int(d["cost"]), int(d["slack"]),
                            int(d["flags"]), lam))
            for h in range(self.H):
                self.sq[h] = deque(e for e in self.sq[h] if id(e) not in committed)
        self.ticks += 1
        return out
