"""Auxiliary subsystems on the GPU: per-call statistics (JSONL), the
bounds-checked build (-DLLAMA_CHECK) on the parity workloads, and NVTX ranges
compiled into the library."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2102_01887_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.gpu
def test_stats_file_records_every_blocking_call(cuda_device, tmp_path):
    from paper_2102_01887_b300 import build, llama as L
    build.build()
    p, inv = W.medium(n_inv=5000)
    bad = W.Invocations(np.where(np.arange(inv.n) % 50 == 0, -1, inv.dag).astype(np.int32), inv.op_local,
                        inv.start_us, inv.now_us)
    path = tmp_path / "calls.jsonl"
    with L.Scheduler(p, use_graph=True) as s:
        L.llama_set_stats_file(s.ctx, path)
        s.schedule(inv)
        s.schedule(bad)
        s.schedule(inv)
        L.llama_set_stats_file(s.ctx, None)
        s.schedule(inv)  # not recorded
    rows = [json.loads(line) for line in open(path)]
    assert [r["call"] for r in rows] == [0, 1, 2]
    assert all(r["n_inv"] == inv.n and r["launches"] >= 2 and r["device_us"] > 0 and r["host_us"] > 0
               for r in rows)
    assert [r["invalid"] for r in rows] == [0, int((bad.dag < 0).sum()), 0]
    assert not any(r["timeout"] for r in rows) and rows[0]["graph"] is True
    # what the decisions say, counted on the host: feasible ones, configurations scored
    with L.Scheduler(p, use_graph=True) as s:
        d, _ = s.schedule(inv)
    ncfg = np.diff(p.cfg_off)[p.dag_op_off[inv.dag] + inv.op_local]
    assert rows[0]["feasible"] == int((d["flags"] & L.FLAG_FEASIBLE != 0).sum())
    assert rows[0]["configs_scored"] == int(ncfg.sum())
    valid = bad.dag >= 0
    assert rows[1]["configs_scored"] == int(ncfg[valid].sum())
    assert rows[0]["inv_per_s"] > 0 and rows[0]["configs_per_s"] > 0


@pytest.mark.gpu
def test_checked_build_parity(cuda_device):
    from paper_2102_01887_b300 import build
    build.build_check()
    env = dict(os.environ, LLAMA_LIB="check")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_build_parity.py")], env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "no bounds check failed" in r.stdout


def test_checked_build_compiles_and_says_so():
    import ctypes
    from paper_2102_01887_b300 import build
    so = build.build_check()
    assert ctypes.CDLL(so).llama_check_build() == 1
    assert ctypes.CDLL(build.build()).llama_check_build() == 0


def test_nvtx_ranges_are_compiled_in():
    from paper_2102_01887_b300 import build
    so = build.build()
    text = open(so, "rb").read()
    # the range names (distinct from every exported symbol name)
    for name in (b"llama:schedule\0", b"llama:schedule_async\0", b"llama:set_profiles\0", b"llama:feedback\0",
                 b"llama:loop_tick\0"):
        assert name in text, name


@pytest.mark.gpu
def test_measured_ceilings_run_and_are_plausible(cuda_device):
    """The micro-benchmarks behind the bench line's denominators: the scan's
    instruction mix runs below one configuration per integer ALU lane per clock
    on every SM, and the bucketing kernel's count atomics alone take longer than
    the same loads and stores without them."""
    import torch
    from paper_2102_01887_b300 import build, llama as L
    build.build()
    sms = torch.cuda.get_device_properties(cuda_device).multi_processor_count
    lane_rate = sms * 64 * 2.2e9  # integer ALU lanes x a clock above the maximum
    for mode in (L.MODE_COST_FIRST, L.MODE_ALPHA):
        sps = L.llama_alu_peak(cuda_device, mode)
        assert 0.1 * lane_rate < sps < lane_rate, (mode, sps)
    atomic_us, stream_us = L.llama_count_rate(cuda_device, 1 << 20, 8368)
    assert 0 < stream_us < atomic_us < 1e4, (atomic_us, stream_us)
    with pytest.raises(L.LlamaError):
        L.llama_count_rate(cuda_device, 0, 8368)
