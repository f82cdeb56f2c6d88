"""The device-resident serving loop (early speculation and late commit, Section
4.3; priority-based commit, Section 4.4) against the oracle's sequential
simulation (oracle/loop.py): every record of every tick -- speculative
decisions, rejections, commits and their order -- bit-exact, and the queueing
times the device holds equal to the simulation's.  Each speculative decision is
also the one a scheduling call of that invocation alone gives under that
tick's queueing time (the same alone and in the mix)."""
import numpy as np
import pytest

import oracle
from oracle.loop import LoopOracle
from paper_2102_01887_b300 import workloads as W
from tests.test_oracle_loop import HAND_QUEUES, HAND_TICKS, TWO_OP_TICKS, micro_problem, two_op_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L(cuda_device):
    from paper_2102_01887_b300 import build, llama
    build.build()
    llama.load()
    return llama


def as_records(res) -> list:
    d = res["decision"]
    return [(int(res["id"][k]), int(res["kind"][k]), int(res["tick"][k]), int(d["cfg"][k]), int(d["lat"][k]),
             int(d["cost"][k]), int(d["slack"][k]), int(d["flags"][k]), int(res["backend"][k]))
            for k in range(res.shape[0])]


def requests(L, reqs):
    r = np.zeros(len(reqs), L.LOOP_REQUEST_DTYPE)
    for k, (i, d, o, st) in enumerate(reqs):
        r[k] = (i, d, o, st)
    return r


def run_device(L, p, script, slots, cq, max_admit=1024, mode=0, alpha=(1, 1), ring=1 << 14):
    out = []
    with L.Scheduler(p, mode=mode, alpha=alpha) as s, \
            L.Loop(s, slots=slots, ring=ring, results=1 << 16, max_admit=max_admit, cq_cap=cq) as lp:
        states = []
        for reqs, now, disp in script:
            assert lp.submit(requests(L, reqs)) == L.OK
            lp.tick(now, disp)
            lp.sync()
            out.append(as_records(lp.poll()))
            states.append(lp.state())
    return out, states


def test_hand_scenarios(L):
    got, states = run_device(L, micro_problem(), [(r, n, d) for r, n, d, _ in HAND_TICKS], slots=10, cq=(1, 1))
    for t, ((_, _, _, want), (q, sq, cq), st) in enumerate(zip(HAND_TICKS, HAND_QUEUES, states)):
        assert got[t] == want, t
        assert st["q_us"] == list(q) and st["sq_len"] == list(sq) and st["cq_len"] == list(cq), t
    got, _ = run_device(L, two_op_problem(), [(r, n, d) for r, n, d, _ in TWO_OP_TICKS], slots=10, cq=(2, 2))
    assert got == [want for _, _, _, want in TWO_OP_TICKS]


def random_script(p, inv, seed, ticks, burst=500, max_dispatch=30):
    rng = np.random.default_rng(seed)
    now, k, script = int(inv.now_us) - 200_000, 0, []
    for _ in range(ticks):
        n = min(int(rng.integers(0, burst)), inv.n - k)
        reqs = [(k + j, int(inv.dag[k + j]), int(inv.op_local[k + j]), int(inv.start_us[k + j]) - 300_000)
                for j in range(n)]
        for j in range(0, n, 97):  # some invalid requests
            reqs[j] = (reqs[j][0], -1, 0, 0)
        k += n
        script.append((reqs, now, [int(x) for x in rng.integers(0, max_dispatch, p.n_hw)]))
        now += int(rng.integers(0, 40_000))
    return script


CASES = {
    "medium_cost_first": (lambda: W.medium(n_inv=6000), 0, (1, 1), (40, 24, 16), 3000),
    "medium_alpha": (lambda: W.medium(n_inv=6000), 1, (3, 2), (40, 24, 16), 3000),
    # Zipf-sized configuration spaces up to 8,192, tight slots (admission waits)
    "batched_tight_slots": (lambda: W.batched(n_inv=6000, n_dags=24), 0, (1, 1), (8, 8, 8), 600),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_random_scripts_match_the_oracle(L, case):
    make, mode, alpha, cq, slots = CASES[case]
    p, inv = make()
    script = random_script(p, inv, 11, ticks=14)
    got, states = run_device(L, p, script, slots=slots, cq=cq, mode=mode, alpha=alpha)
    lo = LoopOracle(p, slots=slots, max_admit=1024, cq_cap=cq, mode=mode, alpha=alpha)
    n_commit = 0
    for t, ((reqs, now, disp), g, st) in enumerate(zip(script, got, states)):
        lo.submit(reqs)
        want = lo.tick(now, disp)
        assert g == want, (case, t, next(((a, b) for a, b in zip(g, want) if a != b), None), len(g), len(want))
        assert st["q_us"] == lo.queueing_time().tolist(), t
        assert st["sq_len"] == [len(x) for x in lo.sq] and st["cq_len"] == [len(x) for x in lo.cq], t
        n_commit += sum(1 for r in g if r[1] == oracle.loop.COMMITTED)
    assert n_commit > 0 and states[-1]["results_dropped"] == 0

    # the same alone and in the mix: the speculative decisions of a tick equal
    # single-invocation calls under that tick's queueing time
    with L.Scheduler(p, mode=mode, alpha=alpha) as s:
        for t in (1, 5, 9):
            reqs, now, _ = script[t]
            spec = {r[0]: r for r in got[t] if r[1] == oracle.loop.SPECULATED}
            L.llama_set_queue(s.ctx, lo.q_log[t][0])
            for i, d, o, st in reqs[:40]:
                if i not in spec:
                    continue
                one = W.Invocations(np.asarray([d], np.int32), np.asarray([o], np.int32),
                                    np.asarray([st], np.int64), now)
                dec, rc = s.schedule(one)
                assert rc == L.OK
                r = spec[i]
                assert (int(dec["cfg"][0]), int(dec["lat"][0]), int(dec["cost"][0]), int(dec["slack"][0]),
                        int(dec["flags"][0])) == r[3:8]


def test_ring_backpressure_and_state(L):
    p, inv = W.medium(n_inv=64)
    with L.Scheduler(p) as s, L.Loop(s, slots=64, ring=8, results=256, max_admit=4, cq_cap=(2, 2, 2)) as lp:
        reqs = requests(L, [(k, int(inv.dag[k]), int(inv.op_local[k]), int(inv.start_us[k])) for k in range(9)])
        assert lp.submit(reqs) == L.EAGAIN  # nine do not fit a ring of eight
        assert lp.submit(reqs[:8]) == L.OK
        assert lp.submit(reqs[8:]) == L.EAGAIN
        lp.tick(inv.now_us)  # admits four (max_admit)
        lp.sync()
        assert lp.submit(reqs[8:]) == L.OK  # four places came free
        st = lp.state()
        assert st["admitted"] == 4 and st["submitted"] == 9 and st["ticks"] == 1
        recs = lp.poll()
        assert sorted(recs["id"][recs["kind"] == L.LOOP_SPECULATED].tolist()) == [0, 1, 2, 3]


def test_driver_thread_serves_every_request(L):
    """The library's driver thread runs the ticks while this thread submits and
    polls: every valid request is speculated and committed once, invalid ones
    are rejected, each decision is its configuration's profile entry with a
    consistent backend, and with every commit queue dispatched whole each tick
    the loop ends empty with every slot free (one more tick after the driver
    stops dispatches the commits of its last tick)."""
    import time
    p, inv = W.medium(n_inv=20_000)
    req = np.zeros(inv.n, L.LOOP_REQUEST_DTYPE)
    req["id"] = np.arange(inv.n)
    req["dag"], req["op_local"], req["start_us"] = inv.dag, inv.op_local, inv.start_us
    req["dag"][::211] = -1
    n_bad = int((req["dag"] < 0).sum())
    seen = {L.LOOP_SPECULATED: [], L.LOOP_COMMITTED: [], L.LOOP_REJECTED: []}
    recs = []
    with L.Scheduler(p) as s, L.Loop(s, slots=4096, ring=1 << 14, results=1 << 16, max_admit=512,
                                     cq_cap=(32, 32, 32)) as lp:
        lp.start(inv.now_us, 2)
        k, t0 = 0, time.time()
        while len(seen[L.LOOP_COMMITTED]) + len(seen[L.LOOP_REJECTED]) < inv.n and time.time() - t0 < 60:
            if k < inv.n and lp.submit(req[k:k + 1000]) == L.OK:
                k = min(inv.n, k + 1000)
            r = lp.poll()
            recs.append(r)
            for kind in seen:
                seen[kind].extend(r["id"][r["kind"] == kind].tolist())
        lp.stop()
        lp.tick(inv.now_us + 10**7, [2**31 - 1] * p.n_hw)
        lp.sync()
        st = lp.state()
    assert sorted(seen[L.LOOP_REJECTED]) == sorted(np.flatnonzero(req["dag"] < 0).tolist())
    good = sorted(np.flatnonzero(req["dag"] >= 0).tolist())
    assert sorted(seen[L.LOOP_SPECULATED]) == good and sorted(seen[L.LOOP_COMMITTED]) == good
    assert st["rejected"] == n_bad and st["committed"] == inv.n - n_bad
    assert st["free_slots"] == 4096 and not any(st["sq_len"]) and not any(st["cq_len"])
    r = np.concatenate(recs)
    r = r[r["kind"] != L.LOOP_REJECTED]
    ids = r["id"]
    g = p.dag_op_off[inv.dag[ids]] + inv.op_local[ids]
    d = r["decision"]
    assert (d["cfg"] >= 0).all() and (d["cfg"] < np.diff(p.cfg_off)[g]).all()
    assert np.array_equal(d["lat"], p.lat_us[p.cfg_off[g] + d["cfg"]])
    assert np.array_equal(d["cost"], p.cost_nd[p.cfg_off[g] + d["cfg"]])
    hw = p.hw_off.reshape(p.n_ops, p.n_hw + 1)
    lam = (hw[g][:, 1:p.n_hw] <= d["cfg"][:, None]).sum(axis=1)
    assert np.array_equal(r["backend"], lam)
    assert np.array_equal(d["flags"] & 1, (d["lat"] < d["slack"]).astype(np.int32))


def test_native_arrival_process_sees_every_record(L):
    """llama_loop_run_arrivals submits requests as their arrival times come and
    polls on the calling thread: every valid request's speculative record comes
    no earlier than its arrival and its commit record no earlier than that, an
    invalid one is rejected (both times at once), the loop ends with every
    slot back; ids that are not id0 + k are refused."""
    p, inv = W.medium(n_inv=5_000)
    n = inv.n
    req = np.zeros(n, L.LOOP_REQUEST_DTYPE)
    req["id"] = 1000 + np.arange(n)
    req["dag"], req["op_local"], req["start_us"] = inv.dag, inv.op_local, inv.start_us
    req["dag"][::97] = -1
    arrive = np.cumsum(np.random.default_rng(4).exponential(1e9 / 2e5, n)).astype(np.int64)  # 2e5 per second
    with L.Scheduler(p) as s, L.Loop(s, slots=4096, ring=1 << 14, results=1 << 16, max_admit=512,
                                     cq_cap=(32, 32, 32)) as lp:
        lp.start(inv.now_us, 2)
        spec, com = lp.run_arrivals(req, arrive, timeout_s=30.0)
        lp.stop()
        lp.tick(inv.now_us + 10**7, [2**31 - 1] * p.n_hw)
        lp.sync()
        st = lp.state()
        bad = req.copy()
        bad["id"][3] += 1
        with pytest.raises(L.LlamaError):
            lp.start(inv.now_us, 2)
            try:
                lp.run_arrivals(bad, arrive)
            finally:
                lp.stop()
    assert (spec >= 0).all() and (com >= spec).all()
    assert (spec >= arrive).all()
    rej = req["dag"] < 0
    assert (spec[rej] == com[rej]).all()
    assert st["rejected"] == int(rej.sum()) and st["committed"] == n - int(rej.sum())
    assert st["free_slots"] == 4096
