"""llama_schedule_static, the allocation-free entry point, against llama_schedule.

Callers that cannot let the library allocate device memory during a call (a
serving loop whose memory is carved up front, a latency-bound loop that cannot
take the CUDA allocator's implicit synchronisation) use llama_schedule_static,
whose scratch is one fixed device array.  Its decisions must equal those of
the allocating entry point bit for bit, on consecutive calls that share (and
inherit) that array.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2102_01887_b300 import workloads as W

pytestmark = pytest.mark.gpu

FIELDS = ("cfg", "lat", "cost", "slack", "flags")


@pytest.mark.parametrize("method", [0, 1], ids=["scan", "staircase"])
def test_static_scratch_matches_allocating_entry_point(cuda_device, method):
    import torch

    from paper_2102_01887_b300 import build, llama as L
    build.build()
    lib = L.load()
    dev = torch.device("cuda", cuda_device)
    p, inv = W.medium()  # 65,536 invocations: the largest size the static array takes
    sub = inv.subset(np.arange(0, inv.n, 5))
    with L.Scheduler(p, device=cuda_device, method=method) as s:
        stream = torch.cuda.Stream(device=dev)
        for case in (inv, sub, inv):  # consecutive calls: a smaller one in between
            expected, rc = s.schedule(case)  # the allocating entry point
            assert rc == L.OK
            dag = torch.from_numpy(case.dag).to(dev)
            opl = torch.from_numpy(case.op_local).to(dev)
            st = torch.from_numpy(case.start_us).to(dev)
            for _ in range(2):  # two calls in a row on the same array
                out = torch.full((case.n * 24,), 0xA5, dtype=torch.uint8, device=dev)
                rc = lib.llama_schedule_static(
                    s.ctx, case.n, dag.data_ptr(), opl.data_ptr(), st.data_ptr(), case.now_us,
                    out.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
                assert rc == L.OK, L.llama_last_error(s.ctx)
                stream.synchronize()
                got = out.cpu().numpy().view(L.DECISION_DTYPE)
                for k in FIELDS:
                    assert np.array_equal(got[k], expected[k]), k

        # sizes beyond the array are rejected before anything runs
        big = L.STATIC_MAX_INV + 1
        rc = lib.llama_schedule_static(s.ctx, big, dag.data_ptr(), opl.data_ptr(), st.data_ptr(),
                                       inv.now_us, out.data_ptr(), None)
        assert rc == L.EINVAL
        assert "LLAMA_STATIC_MAX_INV" in L.llama_last_error(s.ctx)


def test_static_rejects_too_many_operations(cuda_device):
    from paper_2102_01887_b300 import build, llama as L
    build.build()
    lib = L.load()
    p, inv = W.batched(n_inv=1024)  # 8,368 operations > LLAMA_STATIC_MAX_OPS
    assert p.n_ops > L.STATIC_MAX_OPS
    with L.Scheduler(p, device=cuda_device) as s:
        rc = lib.llama_schedule_static(s.ctx, 0, None, None, None, inv.now_us, None, None)
        assert rc == L.EINVAL
        assert "LLAMA_STATIC_MAX_OPS" in L.llama_last_error(s.ctx)


@pytest.mark.parametrize("tuning", [(16, 2, 0, 1), (4, 1, 0, 1), (128, 4, 0, 2)],
                         ids=["default", "256-lanes", "8-lanes-two-stages"])
def test_static_searches_unstaged_latencies_like_the_count_pass(cuda_device, tuning):
    """Ops of 8,192 configurations have more distinct latencies than the scoring
    kernel stages.  The allocating entry point counts them below each slack in a
    separate pass; the allocation-free one, whose array has no room for those
    counts, searches them inside the scoring kernel.  Both must give the oracle's
    decisions, under launch schedules with 32-lane and narrower searches."""
    import torch

    import oracle
    from paper_2102_01887_b300 import build, llama as L
    build.build()
    lib = L.load()
    dev = torch.device("cuda", cuda_device)
    p, inv = W.batched_large(n_dags=32, n_inv=8192)
    assert p.n_ops <= L.STATIC_MAX_OPS
    exp, rc_o = oracle.schedule(p, inv)
    assert rc_o == 0
    with L.Scheduler(p, device=cuda_device) as s:
        L.llama_set_tuning(s.ctx, *tuning)
        got, rc = s.schedule(inv)
        assert rc == L.OK
        assert L.llama_last_launch_count(s.ctx) == 3  # bucketing, count pass, scoring
        dag = torch.from_numpy(inv.dag).to(dev)
        opl = torch.from_numpy(inv.op_local).to(dev)
        st = torch.from_numpy(inv.start_us).to(dev)
        stream = torch.cuda.Stream(device=dev)
        for _ in range(2):
            out = torch.full((inv.n * 24,), 0xA5, dtype=torch.uint8, device=dev)
            rc = lib.llama_schedule_static(s.ctx, inv.n, dag.data_ptr(), opl.data_ptr(), st.data_ptr(),
                                           inv.now_us, out.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
            assert rc == L.OK, L.llama_last_error(s.ctx)
            stream.synchronize()
            got_static = out.cpu().numpy().view(L.DECISION_DTYPE)
            for k in FIELDS:
                assert np.array_equal(got[k], exp[k]), k
                assert np.array_equal(got_static[k], exp[k]), k
