"""The autotuner keeps results unchanged and applies its choice."""
import numpy as np
import pytest

import oracle
from paper_2102_01887_b300 import workloads as W

pytestmark = pytest.mark.gpu


def test_autotune_picks_a_schedule_and_results_stay_exact(cuda_device):
    import torch

    from paper_2102_01887_b300 import build, llama as L
    from paper_2102_01887_b300.autotune import autotune
    build.build()
    p, inv = W.medium()
    sub = inv.subset(np.arange(0, inv.n, 4))
    dev = torch.device("cuda", cuda_device)
    with L.Scheduler(p, use_graph=True) as s:
        dag = torch.from_numpy(sub.dag).to(dev)
        opl = torch.from_numpy(sub.op_local).to(dev)
        st = torch.from_numpy(sub.start_us).to(dev)
        out = torch.zeros(sub.n * 24, dtype=torch.uint8, device=dev)
        res = autotune(s.ctx, dag, opl, st, sub.now_us, out, lanes=(8, 32), ipts=(1, 2), reps=2)
        # 2 lanes x 2 ipt x 2 stagings for each of 4,096 and 8,192 staged
        # distinct latencies, then 4 and 3 scoring CTAs per SM for the fastest;
        # no count-pass trials: every op's distinct latencies are staged by the
        # scoring kernel
        assert len(res["trials"]) == 18 and res["best"]["ms"] > 0
        assert [t["dlat_stage"] for t in res["trials"][:16]] == [4096] * 8 + [8192] * 8
        assert [t.get("ctas_per_sm") for t in res["trials"][16:]] == [4, 3]
        assert res["best"]["dlat_stage"] in (4096, 8192)
        assert res["best"]["count_pass"] == L.COUNT_PASS_AUTO
        assert res["best"]["ctas_per_sm"] in (0, 4, 3)
        out.zero_()
        L.llama_schedule_async(s.ctx, dag, opl, st, sub.now_us, out)
        torch.cuda.synchronize()
    got = out.cpu().numpy().view(L.DECISION_DTYPE)
    exp, _ = oracle.schedule(p, sub)
    for k in ("cfg", "lat", "cost", "slack", "flags"):
        assert np.array_equal(got[k], exp[k]), k


def test_autotune_chooses_the_count_pass_and_results_stay_exact(cuda_device):
    import torch

    from paper_2102_01887_b300 import build, llama as L
    from paper_2102_01887_b300.autotune import autotune
    build.build()
    p, inv = W.batched_large(n_dags=16, n_inv=4096)  # every op beyond the staged latencies
    dev = torch.device("cuda", cuda_device)
    with L.Scheduler(p, use_graph=True) as s:
        dag = torch.from_numpy(inv.dag).to(dev)
        opl = torch.from_numpy(inv.op_local).to(dev)
        st = torch.from_numpy(inv.start_us).to(dev)
        out = torch.zeros(inv.n * 24, dtype=torch.uint8, device=dev)
        res = autotune(s.ctx, dag, opl, st, inv.now_us, out, lanes=(32,), ipts=(1,), stages=(1,), ctas_per_sm=(0,),
                       dlat_stage=(4096,), reps=2)
        assert [t.get("count_pass") for t in res["trials"]] == [None, L.COUNT_PASS_ON, L.COUNT_PASS_OFF]
        assert res["best"]["ms"] == min(t["ms"] for t in res["trials"])
        out.zero_()
        L.llama_schedule_async(s.ctx, dag, opl, st, inv.now_us, out)
        torch.cuda.synchronize()
        assert L.llama_last_launch_count(s.ctx) == (2 if res["best"]["count_pass"] == L.COUNT_PASS_OFF else 3)
    got = out.cpu().numpy().view(L.DECISION_DTYPE)
    exp, _ = oracle.schedule(p, inv)
    for k in ("cfg", "lat", "cost", "slack", "flags"):
        assert np.array_equal(got[k], exp[k]), k
