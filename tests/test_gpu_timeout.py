"""Bounded device waits that give up (failure detection without a GPU fault).

The bucketing kernel's grid barriers poll a bounded number of times.  With the
limit set to 0 every barrier gives up at once -- no fault, no hang, just the
give-up path.  Every entry point must then decide nothing from a bucket
layout that was never finished: every valid invocation comes back with
cfg = -1 and LLAMA_FLAG_TIMEOUT, invalid ones stay flagged invalid, and the
give-up is reported (LLAMA_ETIMEOUT from llama_schedule, the timeout word of
llama_ws_status and llama_static_status).  With the default limit restored the
next calls on the same scratch equal the oracle again.
"""
import ctypes

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


def with_invalid(inv, every=97):
    """A copy of inv with every `every`-th invocation given a DAG id that does not exist."""
    dag = inv.dag.copy()
    dag[::every] = -1
    return W.Invocations(dag, inv.op_local.copy(), inv.start_us.copy(), inv.now_us)


CASES = {
    # profiles of at most 1,024 ops: one grid barrier
    "medium": lambda: W.medium(n_inv=20_000),
    # more ops: three grid barriers
    "batched": lambda: W.batched(n_inv=50_000, n_dags=64),
    # 8,192-configuration tables: the count pass runs between bucketing and scoring
    "batched_large": lambda: W.batched_large(n_dags=48, n_inv=6000),
}


def check_not_decided(L, got, inv):
    bad = inv.dag < 0
    assert (got["cfg"] == -1).all()
    assert (got["flags"][~bad] == L.FLAG_TIMEOUT).all()
    assert (got["flags"][bad] == L.FLAG_INVALID).all()


def same(a, b):
    for f in FIELDS:
        assert np.array_equal(a[f], b[f]), f


@pytest.mark.parametrize("use_graph", [False, True], ids=["direct", "graph"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_barrier_give_up_decides_nothing_and_recovers(L, case, use_graph):
    import torch
    p, inv = CASES[case]()
    inv = with_invalid(inv)
    n_bad = int((inv.dag < 0).sum())
    exp, rc_o = oracle.schedule(p, inv)
    assert rc_o == oracle.EINVAL
    lib = L.load()
    dev = torch.device("cuda", 0)
    d_dag = torch.from_numpy(inv.dag).to(dev)
    d_opl = torch.from_numpy(inv.op_local).to(dev)
    d_st = torch.from_numpy(inv.start_us).to(dev)
    stream = torch.cuda.Stream(device=dev)
    sp = ctypes.c_void_p(stream.cuda_stream)
    with L.Scheduler(p, use_graph=use_graph) as s:
        for limit, timed_out in ((0, True), (L.WAIT_LIMIT_DEFAULT, False), (0, True), (L.WAIT_LIMIT_DEFAULT, False)):
            L.llama_set_wait_limit(s.ctx, limit)
            # blocking entry point, host buffers
            out = np.full(inv.n, -7, L.DECISION_DTYPE)
            rc = lib.llama_schedule(s.ctx, inv.n, inv.dag.ctypes.data, inv.op_local.ctypes.data,
                                    inv.start_us.ctypes.data, inv.now_us, out.ctypes.data)
            if timed_out:
                assert rc == L.ETIMEOUT, L.llama_last_error(s.ctx)
                check_not_decided(L, out, inv)
            else:
                assert rc == L.EINVAL  # the invalid invocations
                same(out, exp)
            # a workspace on another stream, status read back
            ws = ctypes.c_void_p()
            assert lib.llama_ws_create(s.ctx, inv.n, ctypes.byref(ws)) == L.OK
            try:
                o = torch.full((inv.n * 24,), 0x5A, dtype=torch.uint8, device=dev)
                assert lib.llama_schedule_ws_async(s.ctx, ws, inv.n, d_dag.data_ptr(), d_opl.data_ptr(),
                                                   d_st.data_ptr(), inv.now_us, o.data_ptr(), sp) == L.OK
                stream.synchronize()
                n_inv_bad, tmo = ctypes.c_int64(-1), ctypes.c_int32(-1)
                assert lib.llama_ws_status(ws, ctypes.byref(n_inv_bad), ctypes.byref(tmo)) == L.OK
                got = o.cpu().numpy().view(L.DECISION_DTYPE)
                assert tmo.value == int(timed_out) and n_inv_bad.value == n_bad
                if timed_out:
                    check_not_decided(L, got, inv)
                else:
                    same(got, exp)
            finally:
                lib.llama_ws_destroy(ws)
            # the allocation-free entry point (its limits: 65,536 invocations, 4,096 ops)
            if inv.n <= L.STATIC_MAX_INV and p.n_ops <= L.STATIC_MAX_OPS:
                o = torch.full((inv.n * 24,), 0x5A, dtype=torch.uint8, device=dev)
                L.llama_schedule_static(s.ctx, d_dag, d_opl, d_st, inv.now_us, o, stream)
                n_static_bad, tmo = L.llama_static_status(s.ctx, stream)
                got = o.cpu().numpy().view(L.DECISION_DTYPE)
                assert tmo == int(timed_out) and n_static_bad == n_bad
                if timed_out:
                    check_not_decided(L, got, inv)
                else:
                    same(got, exp)


def test_wait_limit_range(L):
    p, _ = W.tiny()
    with L.Scheduler(p) as s:
        lib = L.load()
        assert lib.llama_set_wait_limit(s.ctx, -1) == L.EINVAL
        assert lib.llama_set_wait_limit(s.ctx, L.WAIT_LIMIT_DEFAULT + 1) == L.EINVAL
        assert lib.llama_set_wait_limit(s.ctx, 3) == L.OK
