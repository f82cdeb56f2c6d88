"""Workspace calls on page-locked host arrays (llama_schedule_ws_async): inputs
read in place by the kernels or copied by the copy engine first, decisions
copied back on the caller's stream; two calls in flight on two streams, each
equal to the oracle's decisions; pageable host memory refused."""
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


@pytest.mark.parametrize("inputs", [0, 1], ids=["in_place", "copied"])
def test_host_arrays_two_calls_in_flight(L, inputs):
    import torch
    p, inv = W.medium(n_inv=20_000)
    halves = [inv.subset(np.arange(0, inv.n, 2)), inv.subset(np.arange(1, inv.n, 2))]
    lib = L.load()
    with L.Scheduler(p) as s:
        ws = [ctypes.c_void_p(), ctypes.c_void_p()]
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        pinned = []
        outs = []
        try:
            for w in ws:
                assert lib.llama_ws_create(s.ctx, 10_000, ctypes.byref(w)) == L.OK
                assert lib.llama_ws_set_inputs(w, inputs) == L.OK
            assert lib.llama_ws_set_inputs(ws[0], 2) == L.EINVAL
            for h in halves:
                arrs = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (h.dag, h.op_local, h.start_us)]
                pinned.append(arrs)
                outs.append(torch.zeros(h.n * 24, dtype=torch.uint8).pin_memory())
            for rep in range(3):  # the second and third rounds reuse the staging buffers
                for k, h in enumerate(halves):
                    outs[k].zero_()
                    rc = lib.llama_schedule_ws_async(s.ctx, ws[k], h.n, *(a.data_ptr() for a in pinned[k]),
                                                     h.now_us, outs[k].data_ptr(), streams[k].cuda_stream)
                    assert rc == L.OK
                for st in streams:
                    st.synchronize()
                for k, h in enumerate(halves):
                    got = outs[k].numpy().view(L.DECISION_DTYPE)
                    exp, _ = oracle.schedule(p, h)
                    for f in FIELDS:
                        assert np.array_equal(got[f], exp[f]), (rep, k, f)
            # pageable host memory is refused, for inputs and for the output
            h = halves[0]
            pageable = [np.ascontiguousarray(a) for a in (h.dag, h.op_local, h.start_us)]
            rc = lib.llama_schedule_ws_async(s.ctx, ws[0], h.n, *(a.ctypes.data for a in pageable), h.now_us,
                                             outs[0].data_ptr(), streams[0].cuda_stream)
            assert rc == L.EINVAL
            out_pageable = np.zeros(h.n, L.DECISION_DTYPE)
            rc = lib.llama_schedule_ws_async(s.ctx, ws[0], h.n, *(a.data_ptr() for a in pinned[0]), h.now_us,
                                             out_pageable.ctypes.data, streams[0].cuda_stream)
            assert rc == L.EINVAL
        finally:
            for w in ws:
                if w.value:
                    lib.llama_ws_destroy(w)
