"""The serving loop: continuous batching over several slots.  Every request's
decision must be the same in the mix as alone (bit-exact: integer path) and
equal to the oracle's; batches must overlap on the device."""
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


def requests_from(L, inv, n, n_now=7, seed=0):
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, inv.n, n)
    req = np.zeros(n, L.REQUEST_DTYPE)
    req["id"] = np.arange(n) * 3 + 11
    req["dag"] = inv.dag[idx]
    req["op_local"] = inv.op_local[idx]
    req["start_us"] = inv.start_us[idx]
    req["now_us"] = inv.now_us + 37_000 * rng.integers(0, n_now, n)
    return req


def expected(p, req):
    """The oracle's decision of every request, each against its own now."""
    out = np.zeros(req.shape[0], oracle.DECISION_DTYPE)
    for now in np.unique(req["now_us"]):
        sel = np.flatnonzero(req["now_us"] == now)
        inv = W.Invocations(req["dag"][sel].astype(np.int32), req["op_local"][sel].astype(np.int32),
                            req["start_us"][sel].astype(np.int64), int(now))
        d, _ = oracle.schedule(p, inv)
        out[sel] = d
    return out


def test_results_same_in_the_mix_as_alone(L):
    p, inv = W.medium()
    n = 30_000
    req = requests_from(L, inv, n)
    req["dag"][5] = -1                               # invalid: no such pipeline
    req["start_us"][9] = req["now_us"][9] + 1        # invalid: starts after now
    exp = expected(p, req)
    rng = np.random.default_rng(1)
    got = []
    with L.Scheduler(p) as s, L.Server(s, slots=4, max_batch=2048) as srv:
        k = 0
        while k < n:  # irregular arrivals, polled in between: batches overlap
            m = int(rng.integers(1, 3000))
            assert srv.submit(req[k:k + m]) == L.OK
            k += m
            got.append(srv.poll())
        got.append(srv.drain())
        st = srv.stats()
        # a few requests scheduled alone through the context's own path
        alone_idx = rng.integers(0, n, 100)
        alone = []
        for i in alone_idx:
            one = W.Invocations(np.asarray([req["dag"][i]], np.int32), np.asarray([req["op_local"][i]], np.int32),
                                np.asarray([req["start_us"][i]], np.int64), int(req["now_us"][i]))
            alone.append(s.schedule(one)[0][0])
    res = np.concatenate(got)
    assert res.shape[0] == n
    order = np.argsort(res["id"])
    res = res[order]
    assert np.array_equal(res["id"], req["id"])  # every request exactly once
    for f in FIELDS:
        assert np.array_equal(res["decision"][f], exp[f]), f
    for i, d in zip(alone_idx, alone):
        for f in FIELDS:
            assert res["decision"][f][i] == d[f], (i, f)
    assert res["decision"]["flags"][5] == L.FLAG_INVALID and res["decision"]["flags"][9] == L.FLAG_INVALID
    assert (res["done_ns"] >= res["submit_ns"]).all()
    assert st["completed"] == n and st["batches"] > 10
    assert st["max_in_flight"] >= 2 and st["overlapped"] > 0, st


def test_admission_refuses_beyond_the_queue_bound(L):
    p, inv = W.medium()
    req = requests_from(L, inv, 5000)
    with L.Scheduler(p) as s, L.Server(s, slots=2, max_batch=1024, max_queue=3000) as srv:
        assert srv.submit(req[:2500]) == L.OK
        assert srv.submit(req[2500:5000]) == L.EAGAIN  # would exceed: refused whole
        res = srv.drain()
        assert res.shape[0] == 2500
        assert srv.submit(req[2500:5000]) == L.OK      # room again
        res2 = srv.drain()
        st = srv.stats()
    assert res2.shape[0] == 2500 and st["refused"] == 2500


def test_memory_budget_sets_the_slots(L):
    p, inv = W.medium()
    with L.Scheduler(p) as s, L.Server(s, slots=0, max_batch=1024, memory_budget=64 << 20) as srv:
        st = srv.stats()
    assert 1 <= st["slots"] <= 64


def test_workspaces_run_the_count_pass_side_by_side(L):
    # two workspaces of one context on two streams at once, tables of 8,192
    # configurations (count pass on): each call keeps its counts in its own
    # workspace, and both equal the oracle's decisions
    import ctypes

    import torch
    lib = L.load()
    p, inv = W.batched_large(n_dags=8, n_inv=8192)
    halves = (inv.subset(np.arange(0, inv.n, 2)), inv.subset(np.arange(1, inv.n, 2)))
    exp = [oracle.schedule(p, h)[0] for h in halves]
    with L.Scheduler(p) as s:
        L.llama_set_count_pass(s.ctx, L.COUNT_PASS_ON)
        wss, streams, outs, args = [], [], [], []
        try:
            for h in halves:
                ws = ctypes.c_void_p()
                assert lib.llama_ws_create(s.ctx, h.n, ctypes.byref(ws)) == L.OK, L.llama_last_error(s.ctx)
                wss.append(ws)
                streams.append(torch.cuda.Stream())
                outs.append(torch.full((h.n * 24,), 0xA5, dtype=torch.uint8, device="cuda"))
                args.append([torch.from_numpy(a).cuda() for a in (h.dag, h.op_local, h.start_us)])
            for _ in range(3):  # repeated, the two calls overlapping on the device
                for k, h in enumerate(halves):
                    d, o, st = args[k]
                    rc = lib.llama_schedule_ws_async(s.ctx, wss[k], h.n, d.data_ptr(), o.data_ptr(), st.data_ptr(),
                                                     h.now_us, outs[k].data_ptr(),
                                                     ctypes.c_void_p(streams[k].cuda_stream))
                    assert rc == L.OK, L.llama_last_error(s.ctx)
                torch.cuda.synchronize()
                for k in range(2):
                    got = outs[k].cpu().numpy().view(L.DECISION_DTYPE)
                    for f in FIELDS:
                        assert np.array_equal(got[f], exp[k][f]), (k, f)
        finally:
            for ws in wss:
                lib.llama_ws_destroy(ws)
