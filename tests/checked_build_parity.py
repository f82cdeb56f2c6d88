"""Run in a child process with LLAMA_LIB=check (tests/test_gpu_aux.py): the
bounds-checked build of the library schedules the parity workloads, and every
decision must equal the oracle's with no bounds check failed."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2102_01887_b300 import llama as L  # noqa: E402
from paper_2102_01887_b300 import workloads as W  # noqa: E402

FIELDS = ("cfg", "lat", "cost", "slack", "flags")


def main():
    assert os.environ.get("LLAMA_LIB") == "check"
    lib = L.load()
    assert lib.llama_check_build() == 1, "not the checked build"
    cases = [("tiny", W.tiny(), 0, (1, 1), 0), ("medium", W.medium(n_inv=20_000), 0, (1, 1), 0),
             ("medium_alpha", W.medium(n_inv=20_000), 1, (3, 2), 0),
             ("medium_staircase", W.medium(n_inv=20_000), 0, (1, 1), 1),
             ("batched", W.batched(n_inv=50_000, n_dags=64), 0, (1, 1), 0),
             ("batched_large", W.batched_large(n_dags=16, n_inv=4000), 0, (1, 1), 0),
             ("dag_sizes", W.dag_sizes(), 0, (1, 1), 0)]
    for name, (p, inv), mode, alpha, method in cases:
        dag = inv.dag.copy()
        dag[::101] = -1  # invalid invocations too
        inv = W.Invocations(dag, inv.op_local, inv.start_us, inv.now_us)
        exp, _ = oracle.schedule(p, inv, mode=mode, alpha=alpha)
        with L.Scheduler(p, mode=mode, alpha=alpha, method=method, use_graph=True) as s:
            for _ in range(2):
                got, _ = s.schedule(inv)
                for k in FIELDS:
                    assert np.array_equal(got[k], exp[k]), (name, k)
            assert L.llama_check_word(s.ctx) == 0, name
        print("ok", name, flush=True)
    print("checked build: all parity cases equal the oracle, no bounds check failed")


if __name__ == "__main__":
    main()
