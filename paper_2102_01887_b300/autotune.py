"""Autotuner of the scoring kernel's launch schedule.

The schedule (lanes sharing one invocation, invocations per thread, staging
chunk, staging buffers, whether a count pass precedes the scoring kernel, how
many scoring CTAs share an SM, and how many distinct latencies of an op are
staged beside its table) changes speed, never results (tests check the
latter).  For a given
context and a batch of device-resident invocations, the tuner times every
candidate on that batch -- whole scheduling calls replayed as the caller
would replay them, the L2 cache flushed before each call -- and keeps the
fastest, which it applies with ``llama_set_tuning``.
"""
from __future__ import annotations

import itertools
from typing import Iterable, Optional

from . import llama as L

DEFAULT_LANES_MIN_VECTORS = (4, 8, 16, 32, 64)
DEFAULT_INV_PER_THREAD = (1, 2, 4)
DEFAULT_STAGES = (1, 2)
DEFAULT_CTAS_PER_SM = (0, 4, 3)  # 0: as many as fit
DEFAULT_DLAT_STAGE = (4096, 8192)  # the first is the library default


def time_call(ctx, dag, op_local, start, now: int, out, stream, flush, reps: int = 10) -> float:
    """Device time (ms) of one scheduling call, the L2 flushed before each: the
    mean of reps calls without the fastest and the slowest.  Event timestamps
    advance in steps of about 2 us, so a single call's time, and a median of
    them, only tells schedules apart by whole steps; a mean of readings taken at
    different phases of those steps resolves finer differences."""
    import torch
    times = []
    for r in range(reps + 1):
        with torch.cuda.stream(stream):
            flush.fill_(r & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            L.llama_schedule_async(ctx, dag, op_local, start, now, out, stream)
            e1.record(stream)
        e1.synchronize()
        if r:  # the first call of a setting (re)captures its graph
            times.append(e0.elapsed_time(e1))
    times.sort()
    kept = times[1:-1] if len(times) > 2 else times
    return sum(kept) / len(kept)


def autotune(ctx, dag, op_local, start, now: int, out, stream=None, flush=None,
             lanes: Iterable[int] = DEFAULT_LANES_MIN_VECTORS,
             ipts: Iterable[int] = DEFAULT_INV_PER_THREAD, chunks: Iterable[int] = (0,),
             stages: Iterable[int] = DEFAULT_STAGES, ctas_per_sm: Iterable[int] = DEFAULT_CTAS_PER_SM,
             dlat_stage: Iterable[int] = DEFAULT_DLAT_STAGE, reps: int = 10) -> dict:
    """Sweep the candidates, apply the fastest, return {"best": ..., "trials": [...]}.

    ``chunks``: staging chunk sizes in configurations (0 = the library default);
    ``stages``: staging buffers per CTA (1 or 2); ``dlat_stage``: most distinct
    latencies staged per op, each with the whole grid of the above (the best
    chunk depends on it); ``ctas_per_sm``: caps on the scoring CTAs per SM,
    tried for the fastest schedule (0 = as many as fit).
    """
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    if flush is None:
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dag.device)
    trials = []
    L.llama_set_count_pass(ctx, L.COUNT_PASS_AUTO)
    L.llama_set_score_occupancy(ctx, 0)
    for dls in dlat_stage:
        L.llama_set_dlat_stage(ctx, dls)
        for st, chunk, lmv, ipt in itertools.product(stages, chunks, lanes, ipts):
            L.llama_set_tuning(ctx, lmv, ipt, chunk, st)
            ms = time_call(ctx, dag, op_local, start, now, out, stream, flush, reps)
            trials.append({"lanes_min_vectors": lmv, "inv_per_thread": ipt, "chunk": chunk, "stages": st,
                           "dlat_stage": dls, "ms": ms})
    best = min(trials, key=lambda t: t["ms"])
    L.llama_set_dlat_stage(ctx, best["dlat_stage"])
    L.llama_set_tuning(ctx, best["lanes_min_vectors"], best["inv_per_thread"], best["chunk"], best["stages"])
    # the count pass, forced on and off, against the default for the best
    # schedule -- where it can run at all (forced on, a call launches it)
    best = dict(best, count_pass=L.COUNT_PASS_AUTO)
    for mode in (L.COUNT_PASS_ON, L.COUNT_PASS_OFF):
        L.llama_set_count_pass(ctx, mode)
        ms = time_call(ctx, dag, op_local, start, now, out, stream, flush, reps)
        if mode == L.COUNT_PASS_ON and L.llama_last_launch_count(ctx) < 3:
            break  # no op needs the pass: nothing to choose
        trials.append(dict(best, count_pass=mode, ms=ms))
        if ms < best["ms"]:
            best = trials[-1]
    L.llama_set_count_pass(ctx, best["count_pass"])
    # the CTAs per SM for that schedule
    best = dict(best, ctas_per_sm=0)
    for cap in ctas_per_sm:
        if cap == 0:
            continue
        L.llama_set_score_occupancy(ctx, cap)
        ms = time_call(ctx, dag, op_local, start, now, out, stream, flush, reps)
        trials.append(dict(best, ctas_per_sm=cap, ms=ms))
        if ms < best["ms"]:
            best = trials[-1]
    L.llama_set_score_occupancy(ctx, best["ctas_per_sm"])
    return {"best": best, "trials": trials}
