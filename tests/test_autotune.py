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
        assert len(res["trials"]) == 8 and res["best"]["ms"] > 0  # 2 lanes x 2 ipt x 2 stagings
        out.zero_()
        L.llama_schedule_async(s.ctx, dag, opl, st, sub.now_us, out)
        torch.cuda.synchronize()
    got = out.cpu().numpy().view(L.DECISION_DTYPE)
    exp, _ = oracle.schedule(p, sub)
    for k in ("cfg", "lat", "cost", "slack", "flags"):
        assert np.array_equal(got[k], exp[k]), k
