"""Dumps of a scheduling call as ``.npy`` files, and their bit-exact replay.

``dump(path, problem, inv, decisions, ...)`` writes every array of the
pipelines and profiles (``problem.*.npy``), of the pending invocations
(``inv.*.npy``), the call's decisions (``decisions.npy``, the 24-byte record of
``llama_decision``) and the call's settings (``meta.json``: objective mode,
alpha, method, the time of the call, the queueing times).  ``load(path)``
gives them back with their dtypes and shapes; ``replay(path)`` schedules the
same invocations again through the library and reports whether every field of
every decision is the same.  No counterpart in the paper: this is how a call
seen in a deployment is reproduced offline.
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import llama as L
from .workloads import Invocations, Problem

PROBLEM_ARRAYS = ("dag_op_off", "row_ptr", "col", "slo_us", "cfg_off", "hw_off", "lat_us", "cost_nd", "ref_cfg",
                  "batch", "res", "res_total", "q_us")
INV_ARRAYS = ("dag", "op_local", "start_us")


def dump(path: str, problem, inv, decisions=None, mode: int = L.MODE_COST_FIRST, alpha=(1, 1),
         method: int = L.METHOD_SCAN) -> None:
    os.makedirs(path, exist_ok=True)
    for name in PROBLEM_ARRAYS:
        a = getattr(problem, name)
        if a is not None:
            np.save(os.path.join(path, f"problem.{name}.npy"), np.asarray(a))
    for name in INV_ARRAYS:
        np.save(os.path.join(path, f"inv.{name}.npy"), np.asarray(getattr(inv, name)))
    if decisions is not None:
        np.save(os.path.join(path, "decisions.npy"), np.asarray(decisions, L.DECISION_DTYPE))
    meta = {"n_hw": int(problem.n_hw), "now_us": int(inv.now_us), "mode": int(mode),
            "alpha": [int(alpha[0]), int(alpha[1])], "method": int(method),
            "format": "llama-call-dump-1"}
    with open(os.path.join(path, "meta.json"), "w") as f:
        json.dump(meta, f, indent=1)


def load(path: str):
    """(problem, invocations, decisions or None, meta) of a dump."""
    with open(os.path.join(path, "meta.json")) as f:
        meta = json.load(f)
    arrays = {}
    for name in PROBLEM_ARRAYS:
        fn = os.path.join(path, f"problem.{name}.npy")
        arrays[name] = np.load(fn) if os.path.exists(fn) else None
    p = Problem(n_hw=meta["n_hw"], **arrays)
    inv = Invocations(*(np.load(os.path.join(path, f"inv.{n}.npy")) for n in INV_ARRAYS), meta["now_us"])
    fn = os.path.join(path, "decisions.npy")
    dec = np.load(fn) if os.path.exists(fn) else None
    return p, inv, dec, meta


def replay(path: str, device: int = 0):
    """Schedule a dump's invocations again through the library: (decisions,
    return code, whether they equal the dumped decisions field by field)."""
    p, inv, dec, meta = load(path)
    with L.Scheduler(p, mode=meta["mode"], alpha=tuple(meta["alpha"]), device=device,
                     method=meta["method"]) as s:
        got, rc = s.schedule(inv)
    same = dec is not None and all(np.array_equal(got[k], dec[k]) for k in ("cfg", "lat", "cost", "slack", "flags"))
    return got, rc, same
