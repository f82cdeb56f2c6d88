"""The pins must catch plausible mistakes in the oracle.

Each case plants one mistake into a copy of the oracle's C source (a strict
test made non-strict, a dropped term, a wrong tie-break, a min turned into a
max ...), compiles it on the CPU and checks that at least one pin (the
hand-derived golden example, networkx path enumeration, the independent
staircase selector, the selection invariants) rejects it.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2102_01887_b300 import workloads as W
from tests.problems import load_golden, nx_invocation_slacks, staircase_select

MUTANTS = {
    "feasibility_not_strict": ("(int64_t)p->lat_us[g] < slack_hw[h]",
                               "(int64_t)p->lat_us[g] <= slack_hw[h]"),
    "cost_tie_highest_index": ("take = p->cost_nd[g] < p->cost_nd[first + best]",
                               "take = p->cost_nd[g] <= p->cost_nd[first + best]"),
    "alpha_tie_highest_index": ("obj < best_obj", "obj <= best_obj"),
    "paths_max_not_min": ("if (ps < best) best = ps;",
                          "if (best == INT64_MAX || ps > best) best = ps;"),
    "cp_last_successor_not_max": ("if (cp[col[e]] > best) best = cp[col[e]];",
                                  "best = cp[col[e]];"),
    "cp_excludes_op": ("cp[v] = ref[v] + best;", "cp[v] = best > 0 ? best : ref[v];"),
    "queueing_ignored": ("- t - p->q_us[h];", "- t;"),
    "negative_slack_kept": ("if (R <= 0) return 0;", "if (R <= 0) return R;"),
    "fallback_cheapest_not_fastest": ("take = p->lat_us[g] < p->lat_us[first + best];",
                                      "take = p->cost_nd[g] < p->cost_nd[first + best];"),
    "alpha_drops_r_total": ("* (unsigned __int128)p->res_total[h];", ";"),
    "elapsed_sign_flipped": ("int64_t t = now - start[i];", "int64_t t = start[i] - now;"),
    "ref_is_first_config": ("p->lat_us[p->cfg_off[v] + p->ref_cfg[v]]", "p->lat_us[p->cfg_off[v]]"),
}


def _detect(lib) -> list[str]:
    """Names of the pins the given oracle build fails."""
    failed = []
    g, p, inv = load_golden("amber_worked_example.json")
    for mode, m in (("cost_first", oracle.MODE_COST_FIRST), ("alpha", oracle.MODE_ALPHA)):
        for method in ("critical_path", "paths"):
            d, _ = oracle.schedule(p, inv, mode=m, alpha=tuple(g["alpha"]), method=method, lib=lib)
            exp = g["expected_" + mode]
            if any(d[k].tolist() != exp[k] for k in exp):
                failed.append(f"golden_{mode}_{method}")
        if oracle.slacks(p, inv, method, lib=lib).tolist() != g["expected_slack"]:
            failed.append(f"golden_slack_{method}")
    for seed in range(12):
        p, inv = W.random_small(seed)
        expect = nx_invocation_slacks(p, inv)
        for method in ("critical_path", "paths"):
            if (oracle.slacks(p, inv, method, lib=lib) != expect).any():
                failed.append(f"networkx_slack_{method}_{seed}")
        if (oracle.slacks(p, inv, "paths", lib=lib) != oracle.slacks(p, inv, lib=lib)).any():
            failed.append(f"paths_vs_cp_{seed}")
        for mode, m in (("cost_first", 0), ("alpha", 1)):
            alpha = (1 + seed % 5, 1 + (seed * 7) % 3)
            d, _ = oracle.schedule(p, inv, mode=m, alpha=alpha, lib=lib)
            sl = oracle.slacks(p, inv, lib=lib)
            for i in range(inv.n):
                v = int(p.dag_op_off[inv.dag[i]] + inv.op_local[i])
                if d["cfg"][i] != staircase_select(p, v, sl[i], mode, alpha):
                    failed.append(f"staircase_{mode}_{seed}")
                    break
    return failed


def test_unmutated_oracle_passes_every_pin():
    assert _detect(oracle.load()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(os.path.join(os.path.dirname(oracle.__file__), "llama_oracle.c")).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    so = oracle.build(force=True, src=str(mutated), out=str(tmp_path / "mutant.so"),
                      extra_flags=("-Wno-error",))
    failed = _detect(oracle.load(so))
    assert failed, f"mutant {name} passed every pin"
