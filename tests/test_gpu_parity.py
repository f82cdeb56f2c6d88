"""CUDA path against the CPU oracle, element by element, through the C ABI.

Integer work, so the bar is bit-exact on every field of every decision
(chosen configuration, its latency, cost, slack and flags), on the critical
path and on the slack of every backend.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2102_01887_b300 import workloads as W
from tests.problems import load_golden, single_table_problem

pytestmark = pytest.mark.gpu

FIELDS = ("cfg", "lat", "cost", "slack", "flags")


@pytest.fixture(scope="module")
def L(cuda_device):
    from paper_2102_01887_b300 import build, llama
    build.build()
    llama.load()
    return llama


def assert_same(got, exp, what=""):
    for k in FIELDS:
        bad = np.flatnonzero(got[k] != exp[k])
        assert bad.size == 0, f"{what} field {k}: {bad.size} mismatches, first at {bad[:5]}: " \
                              f"got {got[bad[:5]]} expected {exp[bad[:5]]}"


@pytest.fixture(params=[(0, 0), (0, 1), (1, None)], ids=["scan", "scan_direct", "staircase"])
def method(request, L, monkeypatch):
    """Selection method: the scan of every configuration, bucketed by op (every
    call) or without bucketing (every call up to DIRECT_LIMIT invocations), or
    the staircase."""
    m, direct = request.param
    if direct is not None:
        monkeypatch.setattr(L.Scheduler, "direct_max", L.DIRECT_LIMIT if direct else 0)
    return m


def run_both(L, p, inv, mode=0, alpha=(1, 1), method=0):
    with L.Scheduler(p, mode=mode, alpha=alpha, method=method) as s:
        got, rc = s.schedule(inv)
    exp, rc_o = oracle.schedule(p, inv, mode=mode, alpha=alpha)
    assert rc == rc_o
    return got, exp


# ---------------------------------------------------------------- golden ---

@pytest.mark.parametrize("mode", ["cost_first", "alpha"])
def test_golden_worked_example(L, mode, method):
    g, p, inv = load_golden("amber_worked_example.json")
    m = L.MODE_ALPHA if mode == "alpha" else L.MODE_COST_FIRST
    with L.Scheduler(p, mode=m, alpha=tuple(g["alpha"]), method=method) as s:
        assert s.critical_path().tolist() == g["expected_critical_path"]
        assert s.slack(inv).tolist() == g["expected_slack"]
        d, rc = s.schedule(inv)
    assert rc == L.OK
    for k in FIELDS:
        assert d[k].tolist() == g["expected_" + mode][k], k


# --------------------------------------------------- a1, a2 in isolation ---

@pytest.mark.parametrize("name", ["tiny", "medium", "batched"])
def test_critical_path_and_slack(L, name):
    p, inv = W.WORKLOADS[name]()
    sub = inv.subset(np.arange(min(inv.n, 20000)))
    with L.Scheduler(p) as s:
        assert (s.critical_path() == oracle.critical_path(p)).all()
        assert (s.slack(sub) == oracle.slacks(p, sub)).all()


@pytest.mark.parametrize("mode,alpha", [(0, (1, 1)), (1, (3, 2))])
def test_dags_of_every_size(L, mode, alpha, method):
    # one problem holding DAGs of 1 to 1,500 ops: small DAGs take a warp each in
    # the critical-path pass, mid-sized ones a block with the DAG in shared
    # memory, and the largest go through global memory
    p, inv = W.dag_sizes()
    with L.Scheduler(p, mode=mode, alpha=alpha, method=method) as s:
        assert (s.critical_path() == oracle.critical_path(p)).all()
        assert (s.slack(inv) == oracle.slacks(p, inv)).all()
        got, rc = s.schedule(inv)
    exp, rc_o = oracle.schedule(p, inv, mode=mode, alpha=alpha)
    assert rc == rc_o == 0
    assert_same(got, exp)


@pytest.mark.parametrize("shape", ["chain", "branching"])
def test_slack_division_at_its_extremes(L, shape, method):
    """Algorithm 1's division floor(ref * R / cp) at the edge of its range:
    reference latencies and remaining times within a few thousand of 2^31
    (ref * R just below 2^62) over long paths (cp up to about 2^40), so the
    multiply-high by floor((2^64 - 1) / cp) and its one correction are checked
    where they are tightest; slack, critical path and decisions bit-exact."""
    rng = np.random.default_rng(7 if shape == "chain" else 8)
    n = 600
    top = 2**31 - 2
    if shape == "chain":
        succ = [[v + 1] for v in range(n - 1)] + [[]]
        ref = (top - rng.integers(0, 5000, n)).tolist()
    else:  # random branching over later ops, reference latencies spread over [2^20, 2^31)
        succ = [sorted({int(x) for x in rng.integers(v + 1, n, rng.integers(1, 4))}) if v < n - 1 else []
                for v in range(n)]
        ref = np.minimum(top, np.exp(rng.uniform(np.log(2.0**20), np.log(2.0**31), n))).astype(np.int64).tolist()
    extra = [[(int(rng.integers(0, 3)), int(rng.integers(1, top)), int(rng.integers(0, 2**40)))
              for _ in range(int(rng.integers(1, 6)))] for _ in range(n)]
    p = single_table_problem(succ, ref, slo=2**31 - 1, q=(0, 7, 123_456), extra=extra)
    m = 4000
    ops = rng.integers(0, n, m).astype(np.int32)
    now = 10**12
    start = now - rng.integers(0, 3000, m)
    start[::50] = now - rng.integers(0, 2**31 - 1, start[::50].shape[0])  # some far into their target
    inv = W.Invocations(np.zeros(m, np.int32), ops, start.astype(np.int64), now)
    cp = oracle.critical_path(p)
    assert cp.max() > (2**38 if shape == "chain" else 2**32)
    with L.Scheduler(p, method=method) as s:
        assert np.array_equal(s.critical_path(), cp)
        assert np.array_equal(s.slack(inv).astype(np.int64), oracle.slacks(p, inv))
    got, exp = run_both(L, p, inv, method=method)
    assert_same(got, exp, shape)


@pytest.mark.parametrize("seed", range(20))
def test_slack_random_small(L, seed):
    p, inv = W.random_small(seed)
    with L.Scheduler(p) as s:
        assert (s.critical_path() == oracle.critical_path(p)).all()
        assert (s.slack(inv) == oracle.slacks(p, inv)).all()


# ------------------------------------------------------------- full path ---

@pytest.mark.parametrize("seed", range(40))
@pytest.mark.parametrize("mode", [0, 1])
def test_random_small(L, seed, mode, method):
    p, inv = W.random_small(seed, max_cfg=24, n_inv=300)
    got, exp = run_both(L, p, inv, mode, alpha=(1 + seed % 7, 1 + seed % 3), method=method)
    assert_same(got, exp, f"seed {seed}")


def test_tiny(L, method):
    p, inv = W.tiny()
    got, exp = run_both(L, p, inv, method=method)
    assert_same(got, exp)


def test_medium_full(L, method):
    # the benchmark's workload, every invocation
    p, inv = W.medium()
    got, exp = run_both(L, p, inv, method=method)
    assert_same(got, exp)
    assert 0.5 < (got["flags"] & 1).mean() < 1.0  # both branches exercised


def test_medium_alpha(L, method):
    p, inv = W.medium()
    sub = inv.subset(np.arange(0, inv.n, 3))
    got, exp = run_both(L, p, sub, mode=1, alpha=(3, 2), method=method)
    assert_same(got, exp)


@pytest.mark.slow
def test_batched_full(L, method):
    p, inv = W.batched()
    got, exp = run_both(L, p, inv, method=method)
    assert_same(got, exp)


@pytest.mark.slow
def test_batched_full_alpha(L, method):
    """The headline workload in alpha mode (Eq. 1's penalty for missing the
    target, alpha = 3/2), every decision of all 1,048,576 invocations."""
    p, inv = W.batched()
    got, exp = run_both(L, p, inv, mode=1, alpha=(3, 2), method=method)
    assert_same(got, exp)


# ------------------------------------------------------------ edge cases ---

def test_empty_call(L, method):
    p, inv = W.tiny()
    with L.Scheduler(p, method=method) as s:
        d, rc = s.schedule(inv.subset(np.arange(0)))
    assert rc == L.OK and d.shape == (0,)


def test_invalid_invocations_mixed_with_valid(L, method):
    g, p, inv = load_golden("amber_worked_example.json")
    bad = W.Invocations(np.asarray([0, 1, 0, 0, -1, 0], np.int32),
                        np.asarray([1, 0, 4, 2, 0, -3], np.int32),
                        np.asarray([9400, 9400, 9400, 10001, 0, 9400], np.int64), 10000)
    with L.Scheduler(p, method=method) as s:
        d, rc = s.schedule(bad)
    exp, rc_o = oracle.schedule(p, bad)
    assert rc == L.EINVAL == rc_o
    assert_same(d, exp)
    assert d["cfg"].tolist() == [5, -1, -1, -1, -1, -1]


def _with_invalid(inv, every: int):
    """inv with every `every`-th invocation made invalid, by turns: no such DAG,
    an op index past its DAG, a start after now."""
    dag, opl, st = inv.dag.copy(), inv.op_local.copy(), inv.start_us.copy()
    idx = np.arange(0, inv.n, every)
    kind = (idx // every) % 3
    dag[idx[kind == 0]] = -1
    opl[idx[kind == 1]] = 10_000
    st[idx[kind == 2]] = inv.now_us + 1
    return W.Invocations(dag, opl, st, inv.now_us)


@pytest.mark.slow
@pytest.mark.parametrize("shape", ["medium_600k", "batched"])
def test_invalid_invocations_in_every_counting_round(L, shape):
    """Enough invocations that every counting thread of the bucketing kernel
    takes rounds beyond the ones it keeps in registers -- on the one-barrier
    layout (medium: at most 1,024 ops) and the three-barrier one (batched) --
    with invalid invocations spread over all of them: every decision equal to
    the oracle's, the invalid ones flagged, the call's status EINVAL."""
    p, inv = W.medium(n_inv=600_000) if shape == "medium_600k" else W.batched()
    bad = _with_invalid(inv, 37)
    got, exp = run_both(L, p, bad)
    assert_same(got, exp)
    n_bad = len(range(0, inv.n, 37))
    assert int((got["flags"] & L.FLAG_INVALID != 0).sum()) == n_bad
    assert (got["cfg"][::37] == -1).all()


@pytest.mark.parametrize("q", [(0, 7000, 7000), (3000, 0, 3000), (5000, 5000, 5000), (0, 0, 9000)],
                         ids=["last-two", "first-last", "all-equal", "first-two"])
@pytest.mark.parametrize("shape", ["medium", "batched"])
def test_backends_sharing_a_queueing_time(L, shape, q):
    """Queueing times equal on some backends and not on others (equal ones give
    an invocation equal slacks on those backends): every grouping of three
    backends, on whole-CTA tiles (medium) and on warp tiles too (batched),
    against the oracle."""
    p, inv = W.medium(n_inv=20_000) if shape == "medium" else W.batched(n_inv=200_000)
    p.q_us = np.asarray(q, np.int64)
    got, exp = run_both(L, p, inv)
    assert_same(got, exp)


def test_all_targets_passed(L, method):
    p, inv = W.medium()
    late = W.Invocations(inv.dag, inv.op_local, np.zeros(inv.n, np.int64), inv.now_us)
    got, exp = run_both(L, p, late.subset(np.arange(5000)), method=method)
    assert_same(got, exp)
    assert (got["flags"] == 0).all() and (got["slack"] == 0).all()


def test_all_ties(L, method):
    # identical latency and cost everywhere: the lowest index must win
    p, inv = W.medium()
    p.lat_us[:] = 1000
    p.cost_nd[:] = 7
    got, exp = run_both(L, p, inv.subset(np.arange(3000)), method=method)
    assert_same(got, exp)


def test_single_config_ops_and_single_backend_segments(L, method):
    # ops with one configuration, ops whose configurations all sit on one backend
    p = single_table_problem([[1, 2], [3], [3], []], [10, 20, 30, 40], slo=400,
                             extra=[[], [(2, 5, 100), (2, 4, 100), (2, 4, 50)], [(1, 29, 1)],
                                    [(0, 39, 2), (0, 41, 1)]])
    rng = np.random.default_rng(5)
    n = 500
    inv = W.Invocations(np.zeros(n, np.int32), rng.integers(0, 4, n).astype(np.int32),
                        (10**6 - rng.integers(0, 500, n)).astype(np.int64), 10**6)
    for mode in (0, 1):
        got, exp = run_both(L, p, inv, mode, method=method)
        assert_same(got, exp)


def test_largest_config_space_with_ties(L, method):
    # 8,192 configurations per op (the limit), heavy ties, several tiles per op
    p, inv = W.random_small(3, max_dags=1, max_ops=4, max_cfg=2, n_inv=2000, value_range=5000)
    n = 8192
    rng = np.random.default_rng(9)
    k = p.n_ops
    p.cfg_off = np.arange(0, (k + 1) * n, n, dtype=np.int64)
    cuts = np.sort(rng.integers(0, n, size=(k, 2)), axis=1)
    p.hw_off = np.concatenate([np.zeros((k, 1)), cuts, np.full((k, 1), n)], axis=1).astype(np.int32).ravel()
    p.lat_us = rng.integers(1, 3000, size=k * n).astype(np.int32)
    p.cost_nd = rng.integers(0, 50, size=k * n).astype(np.int64)
    p.ref_cfg = rng.integers(0, n, size=k).astype(np.int32)
    p.batch = rng.integers(1, 4, size=k * n).astype(np.int32)
    p.res = rng.integers(1, 4, size=k * n).astype(np.int32)
    p.slo_us[:] = 20000
    for mode in (0, 1):
        got, exp = run_both(L, p, inv, mode, alpha=(2, 3), method=method)
        assert_same(got, exp)


@pytest.mark.parametrize("n_hw", [1, 2, 8])
def test_backend_counts(L, n_hw, method):
    rng = np.random.default_rng(n_hw)
    p, inv = W.random_small(100 + n_hw, max_cfg=40, n_inv=1000)
    k = p.n_ops
    sizes = np.diff(p.cfg_off)
    hw = []
    for n in sizes:
        cuts = np.sort(rng.integers(0, n + 1, size=n_hw - 1))
        hw.append(np.concatenate([[0], cuts, [n]]))
    p.n_hw = n_hw
    p.hw_off = np.concatenate(hw).astype(np.int32)
    p.q_us = rng.integers(0, 20, size=n_hw).astype(np.int64)
    p.res_total = rng.integers(1, 9, size=n_hw).astype(np.int32)
    assert p.hw_off.shape[0] == k * (n_hw + 1)
    for mode in (0, 1):
        got, exp = run_both(L, p, inv, mode, alpha=(5, 2), method=method)
        assert_same(got, exp)


@pytest.mark.parametrize("n_hw", [5, 8])
def test_count_pass_with_more_than_four_backends(L, n_hw):
    # 8,192-configuration tables split into 5 or 8 backend segments: the count
    # pass's eight-backend variant and the scoring kernel's own searches (pass
    # off) against the oracle, in both objectives
    rng = np.random.default_rng(40 + n_hw)
    p, inv = W.batched_large(n_dags=4, n_inv=2048)
    hw = []
    for n in np.diff(p.cfg_off):
        cuts = np.sort(rng.integers(1, n, size=n_hw - 1))  # the reference configuration stays on backend 0
        hw.append(np.concatenate([[0], cuts, [n]]))
    p.n_hw = n_hw
    p.hw_off = np.concatenate(hw).astype(np.int32)
    p.q_us = rng.integers(0, 100_000, size=n_hw).astype(np.int64)
    p.res_total = rng.integers(1, 9, size=n_hw).astype(np.int32)
    for mode in (0, 1):
        exp, _ = oracle.schedule(p, inv, mode=mode, alpha=(5, 2))
        with L.Scheduler(p, mode=mode, alpha=(5, 2)) as s:
            assert L.load().llama_set_count_pass(s.ctx, 7) == L.EINVAL
            for cp, launches in ((L.COUNT_PASS_ON, 3), (L.COUNT_PASS_OFF, 2)):
                L.llama_set_count_pass(s.ctx, cp)
                got, rc = s.schedule(inv)
                assert rc == L.OK
                assert L.llama_last_launch_count(s.ctx) == launches
                assert_same(got, exp, f"{n_hw} backends, mode {mode}, count pass {cp}")


# ---------------------------------------------------- device-side calls ---

def test_device_pointers_and_async_stream(L, method):
    import torch
    p, inv = W.medium()
    exp, _ = oracle.schedule(p, inv)
    dev = torch.device("cuda:0")
    dag = torch.from_numpy(inv.dag).to(dev)
    opl = torch.from_numpy(inv.op_local).to(dev)
    st = torch.from_numpy(inv.start_us).to(dev)
    with L.Scheduler(p, method=method) as s:
        out = torch.zeros(inv.n * 24, dtype=torch.uint8, device=dev)
        L.llama_schedule(s.ctx, dag, opl, st, inv.now_us, out)  # blocking, device pointers
        got = out.cpu().numpy().view(L.DECISION_DTYPE)
        assert_same(got, exp, "blocking device")
        stream = torch.cuda.Stream()
        out2 = torch.zeros_like(out)
        L.llama_reserve(s.ctx, inv.n)
        for _ in range(3):  # repeated calls reuse the scratch
            L.llama_schedule_async(s.ctx, dag, opl, st, inv.now_us, out2, stream)
        stream.synchronize()
        assert_same(out2.cpu().numpy().view(L.DECISION_DTYPE), exp, "async")
        assert L.llama_last_launch_count(s.ctx) >= 1


def test_pinned_host_inputs(L, method):
    """Page-locked host inputs are read in place by the kernels; pageable ones
    are copied first; the decisions are the same either way, with host or
    device output, and with invalid invocations among them."""
    import torch
    p, inv = W.medium()
    inv = inv.subset(np.arange(0, inv.n, 3))
    inv.dag = inv.dag.copy()
    inv.start_us = inv.start_us.copy()
    inv.dag[5] = -1
    inv.start_us[9] = inv.now_us + 1
    exp, _ = oracle.schedule(p, inv)
    h_dag = torch.from_numpy(inv.dag).pin_memory()
    h_opl = torch.from_numpy(inv.op_local).pin_memory()
    h_st = torch.from_numpy(inv.start_us).pin_memory()
    with L.Scheduler(p, method=method) as s:
        for out in (np.zeros(inv.n, dtype=L.DECISION_DTYPE),
                    torch.zeros(inv.n * 24, dtype=torch.uint8).pin_memory(),
                    torch.zeros(inv.n * 24, dtype=torch.uint8, device="cuda:0")):
            got, rc = L.llama_schedule(s.ctx, h_dag, h_opl, h_st, inv.now_us, out)
            assert rc == L.EINVAL  # the two invalid invocations
            got = got if isinstance(got, np.ndarray) else got.cpu().numpy().view(L.DECISION_DTYPE)
            assert_same(got, exp, "pinned inputs")
        # one pinned, two pageable
        got, _ = L.llama_schedule(s.ctx, h_dag, inv.op_local, inv.start_us, inv.now_us)
        assert_same(got, exp, "mixed inputs")


def test_growing_and_shrinking_batches(L, method):
    p, inv = W.medium()
    exp, _ = oracle.schedule(p, inv)
    with L.Scheduler(p, method=method) as s:
        for n in (17, 65536, 1, 4096, 65535):
            idx = np.arange(n)
            got, rc = s.schedule(inv.subset(idx))
            assert rc == L.OK
            assert_same(got, exp[idx], f"n={n}")


def test_errors(L):
    p, inv = W.tiny()
    ctx = L.llama_create(0, 3)
    try:
        with pytest.raises(L.LlamaError) as e:
            L.llama_schedule(ctx, inv.dag, inv.op_local, inv.start_us, inv.now_us)
        assert e.value.code == L.ENOTREADY
        with pytest.raises(L.LlamaError) as e:  # cycle
            L.llama_set_dags(ctx, [0, 2], [0, 1, 2], [1, 0], [100])
        assert e.value.code == L.EINVAL
        with pytest.raises(L.LlamaError):  # cross-DAG edge
            L.llama_set_dags(ctx, [0, 1, 2], [0, 1, 1], [1], [100, 100])
        with pytest.raises(L.LlamaError):  # latency 0
            L.llama_set_profiles(ctx, [0, 1], [0, 1, 1, 1], [0], [1], [0])
        with pytest.raises(L.LlamaError):  # ref_cfg out of range
            L.llama_set_profiles(ctx, [0, 1], [0, 1, 1, 1], [5], [1], [1])
        with pytest.raises(L.LlamaError):  # more than 8192 configurations
            n = 8193
            L.llama_set_profiles(ctx, [0, n], [0, n, n, n], np.ones(n), np.ones(n), [0])
        with pytest.raises(L.LlamaError):  # negative queueing time
            L.llama_set_queue(ctx, [0, -1, 0])
        with pytest.raises(L.LlamaError) as e:  # tuning before the profiles
            L.llama_set_tuning(ctx, 16, 2, 0, 1)
        assert e.value.code == L.ENOTREADY
        with pytest.raises(L.LlamaError) as e:
            L.llama_set_score_occupancy(ctx, 4)
        assert e.value.code == L.ENOTREADY
        with pytest.raises(L.LlamaError) as e:
            L.llama_set_dlat_stage(ctx, 4096)
        assert e.value.code == L.ENOTREADY
        for bad in ((0, 2, 0, 1), (2048, 2, 0, 1), (16, 3, 0, 1), (16, 2, 12, 1), (16, 2, 8264, 1),
                    (16, 2, 0, 3), (16, 2, 0, 0)):
            with pytest.raises(L.LlamaError) as e:
                L.llama_set_tuning(ctx, *bad)
            assert e.value.code == L.EINVAL, bad
        for bad in (-1, 33):
            with pytest.raises(L.LlamaError) as e:
                L.llama_set_score_occupancy(ctx, bad)
            assert e.value.code == L.EINVAL, bad
        for bad in (0, 8193):
            with pytest.raises(L.LlamaError) as e:
                L.llama_set_dlat_stage(ctx, bad)
            assert e.value.code == L.EINVAL, bad
    finally:
        L.llama_destroy(ctx)


def test_method_switch_and_profile_reload(L):
    # switching methods on one context, and new profiles while the staircase is
    # active (its tables are rebuilt from them)
    import dataclasses
    p, inv = W.medium()
    sub = inv.subset(np.arange(0, inv.n, 5))
    exp, _ = oracle.schedule(p, sub)
    with L.Scheduler(p) as s:
        for m in (1, 0, 1, 1, 0, 1):
            L.llama_set_method(s.ctx, m)
            got, rc = s.schedule(sub)
            assert rc == L.OK
            assert_same(got, exp, f"method {m}")
        rng = np.random.default_rng(4)
        p2 = dataclasses.replace(p, lat_us=(p.lat_us // 2 + rng.integers(0, 50, p.n_cfg)).astype(np.int32) + 1,
                                 cost_nd=p.cost_nd[::-1].copy())
        L.llama_set_profiles(s.ctx, p2.cfg_off, p2.hw_off, p2.lat_us, p2.cost_nd, p2.ref_cfg)
        got, rc = s.schedule(sub)
        exp2, _ = oracle.schedule(p2, sub)
        assert_same(got, exp2, "new profiles")
        with pytest.raises(L.LlamaError) as e:
            L.llama_set_method(s.ctx, 2)
        assert e.value.code == L.EINVAL


# ----------------------------------------------------------- graph replay ---

def test_graph_replay_tracks_now_sizes_and_contents(L, method):
    # one context in graph mode: the call is captured once per argument set and
    # replayed; `now` is patched per call; staging buffers keep host calls on one graph
    import torch
    p, inv = W.medium()
    with L.Scheduler(p, use_graph=True, method=method) as s:
        for k, n in enumerate((65536, 65536, 4096, 4096, 65536)):
            shift = 1000 * k  # later `now`, same elapsed time as before plus the shift
            case = W.Invocations(inv.dag[:n], inv.op_local[:n], inv.start_us[:n], inv.now_us + shift)
            got, rc = s.schedule(case)
            exp, rc_o = oracle.schedule(p, case)
            assert rc == rc_o == L.OK
            assert_same(got, exp, f"call {k}")
        # traced calls on device pointers (direct launches), then untraced replay again
        dev = torch.device("cuda:0")
        dag = torch.from_numpy(inv.dag).to(dev)
        opl = torch.from_numpy(inv.op_local).to(dev)
        st = torch.from_numpy(inv.start_us).to(dev)
        out = torch.zeros(inv.n * 24, dtype=torch.uint8, device=dev)
        stream = torch.cuda.Stream()
        exp, _ = oracle.schedule(p, inv)
        for rep in range(3):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(L.TRACE_EVENTS)]
            with torch.cuda.stream(stream):
                L.llama_set_trace_events(s.ctx, ev)
                L.llama_schedule_async(s.ctx, dag, opl, st, inv.now_us, out, stream)
            stream.synchronize()
            assert all(ev[j].elapsed_time(ev[j + 1]) >= 0 for j in range(L.TRACE_EVENTS - 1))
            assert_same(out.cpu().numpy().view(L.DECISION_DTYPE), exp, f"traced {rep}")
        L.llama_set_trace_events(s.ctx, [])
        out.zero_()
        L.llama_schedule_async(s.ctx, dag, opl, st, inv.now_us, out, stream)
        stream.synchronize()
        assert_same(out.cpu().numpy().view(L.DECISION_DTYPE), exp, "untraced after traced")


# ------------------------------------------------------- launch schedules ---

@pytest.mark.parametrize("tuning", [(1, 1, 0, 1), (4, 2, 0, 1), (16, 4, 0, 1), (64, 2, 0, 1),
                                    (1024, 1, 0, 1), (16, 2, 64, 1), (2, 4, 8, 1), (8, 1, 136, 1),
                                    (1, 1, 0, 2), (16, 2, 0, 2), (32, 1, 0, 2), (64, 4, 0, 2),
                                    (1024, 2, 0, 2), (16, 2, 64, 2), (2, 1, 8, 2), (8, 4, 136, 2)])
def test_tunings_change_no_result(L, tuning):
    # every kernel variant (1/2/4 invocations per thread), lane counts from one
    # to a whole CTA per invocation, and chunked staging of tables larger than
    # the chunk, on ties-heavy random problems and on the benchmark's workload
    p, inv = W.random_small(77, max_cfg=300, n_inv=3000, value_range=200)
    pm, invm = W.medium()
    subm = invm.subset(np.arange(0, invm.n, 7))
    # ops of 8,192 configurations: their distinct latencies are not staged, so
    # they are counted below each slack by the count pass, or (pass off)
    # searched in global memory by groups of 1 to 256 lanes
    pl, invl = W.batched_large(n_dags=4, n_inv=2048)
    for prob, case, passes in ((p, inv, (L.COUNT_PASS_AUTO,)), (pm, subm, (L.COUNT_PASS_AUTO,)),
                               (pl, invl, (L.COUNT_PASS_ON, L.COUNT_PASS_OFF))):
        for mode in (0, 1):
            exp, _ = oracle.schedule(prob, case, mode=mode, alpha=(2, 3))
            for cp in passes:
                with L.Scheduler(prob, mode=mode, alpha=(2, 3)) as s:
                    L.llama_set_tuning(s.ctx, *tuning)
                    L.llama_set_count_pass(s.ctx, cp)
                    got, rc = s.schedule(case)
                assert rc == L.OK
                assert_same(got, exp, f"tuning {tuning} mode {mode} count pass {cp}")


@pytest.mark.parametrize("mode", [0, 1], ids=["cost_first", "alpha"])
def test_warp_tiles_and_occupancy_change_no_result(L, mode):
    # ops of 1..700 configurations on 3 backends: padded tables on both sides
    # of the size a warp scores alone (576 entries cost-first, 456 alpha), so
    # whole-CTA tiles and warp tiles in one call; 108 to 151 invocations per op
    # (ragged warp tiles); every invocations per thread, one and two staging
    # buffers, and 1 to 4 scoring CTAs per SM
    p, inv = W.random_small(5, max_dags=6, max_ops=12, max_cfg=700, n_inv=5000, value_range=400)
    npad = np.diff(p.hw_off.reshape(p.n_ops, p.n_hw + 1), axis=1)
    npad = ((npad + 7) // 8 * 8).sum(axis=1)
    limit = 576 if mode == 0 else 456
    assert (npad <= limit).any() and (npad > limit).any()
    exp, _ = oracle.schedule(p, inv, mode=mode, alpha=(2, 3))
    with L.Scheduler(p, mode=mode, alpha=(2, 3)) as s:
        for tuning, per_sm in (((16, 1, 0, 1), 0), ((16, 2, 0, 1), 0), ((16, 4, 0, 1), 0), ((4, 2, 0, 1), 1),
                               ((64, 2, 0, 1), 2), ((8, 4, 0, 2), 3), ((16, 1, 0, 2), 4), ((16, 2, 64, 1), 0)):
            L.llama_set_tuning(s.ctx, *tuning)
            L.llama_set_score_occupancy(s.ctx, per_sm)
            got, rc = s.schedule(inv)
            assert rc == L.OK
            assert_same(got, exp, f"tuning {tuning} ctas per sm {per_sm}")


@pytest.mark.parametrize("mode", [0, 1], ids=["cost_first", "alpha"])
def test_count_pass_changes_no_result(L, mode):
    # Zipf-sized tables (a few ops beyond the staged distinct latencies, each
    # with many invocations: AUTO leaves the pass off) and all ops at 8,192
    # configurations (AUTO turns it on); every setting gives the oracle's
    # decisions, and the launch count shows whether the pass ran
    cases = ((W.batched(n_inv=65536), 2), (W.batched_large(n_dags=24, n_inv=6000), 3))
    for (prob, case), auto_launches in cases:
        exp, _ = oracle.schedule(prob, case, mode=mode, alpha=(2, 3))
        with L.Scheduler(prob, mode=mode, alpha=(2, 3)) as s:
            for cp, launches in ((L.COUNT_PASS_AUTO, auto_launches), (L.COUNT_PASS_ON, 3),
                                 (L.COUNT_PASS_OFF, 2), (L.COUNT_PASS_ON, 3)):
                L.llama_set_count_pass(s.ctx, cp)
                got, rc = s.schedule(case)
                assert rc == L.OK
                assert L.llama_last_launch_count(s.ctx) == launches, cp
                assert_same(got, exp, f"count pass {cp}")


@pytest.mark.parametrize("mode", [0, 1], ids=["cost_first", "alpha"])
def test_dlat_stage_changes_no_result(L, mode):
    # the distinct latencies staged per op from 1 (almost every op counted by
    # the count pass or searched in global memory) to 8,192 (every op staged),
    # with the pass forced on (launched while some op could have more distinct
    # latencies than are staged, after feedback too) and off, on Zipf-sized
    # and on 8,192-configuration tables
    cases = (W.batched(n_inv=65536), W.batched_large(n_dags=24, n_inv=6000))
    for prob, case in cases:
        exp, _ = oracle.schedule(prob, case, mode=mode, alpha=(2, 3))
        sizes = np.diff(prob.cfg_off)
        dn = np.asarray([np.unique(prob.lat_us[prob.cfg_off[v]:prob.cfg_off[v + 1]]).size
                         for v in range(prob.n_ops)])
        with L.Scheduler(prob, mode=mode, alpha=(2, 3)) as s:
            for stage in (1, 64, 4096, 8192):
                L.llama_set_dlat_stage(s.ctx, stage)
                # staged room: the largest list of at most `stage` entries; the
                # pass is launched (forced on) while some op's configurations
                # exceed it
                staged = dn[dn <= stage]
                cap = (int(staged.max()) + 3) // 4 * 4 if staged.size else 0
                for cp in (L.COUNT_PASS_ON, L.COUNT_PASS_OFF):
                    L.llama_set_count_pass(s.ctx, cp)
                    got, rc = s.schedule(case)
                    assert rc == L.OK
                    launches = 3 if cp == L.COUNT_PASS_ON and sizes.max() > cap else 2
                    assert L.llama_last_launch_count(s.ctx) == launches, (stage, cp)
                    assert_same(got, exp, f"dlat stage {stage} count pass {cp}")


@pytest.fixture(scope="module")
def batched_large():
    return W.batched_large()


@pytest.mark.slow
@pytest.mark.parametrize("mode,alpha", [(0, (1, 1)), (1, (3, 2))])
def test_batched_large_full(L, batched_large, mode, alpha, method):
    # every op at 8,192 configurations (1.6 GB of tables, far beyond L2), about two
    # invocations per op: the HBM-streaming regime, chunked staging, wide groups
    p, inv = batched_large
    got, exp = run_both(L, p, inv, mode=mode, alpha=alpha, method=method)
    assert_same(got, exp)


# ------------------------------------------------------------- small calls ---

def test_small_calls_skip_the_bucketing(L):
    # A call of at most the limit's invocations has no bounded wait (critical
    # paths, then a warp per invocation): with a wait limit of 0 it still
    # decides, one invocation above the limit is bucketed and gives up.  Both
    # sides of the limit, the limit off and at its maximum, and the static
    # entry point with invalid invocations, against the oracle.
    import torch
    lib = L.load()
    p, inv = W.medium(n_inv=4096)
    assert L.Scheduler.direct_max is None  # the library default applies
    with L.Scheduler(p) as s:
        assert lib.llama_set_direct_max(s.ctx, -1) == L.EINVAL
        assert lib.llama_set_direct_max(s.ctx, L.DIRECT_LIMIT + 1) == L.EINVAL
        L.llama_set_wait_limit(s.ctx, 0)
        # (a bucketed call gives up only with two counting blocks or more: over 256 invocations)
        for limit, n, decided in ((None, L.DIRECT_DEFAULT, True), (None, L.DIRECT_DEFAULT + 1, False),
                                  (0, 300, False), (300, 300, True), (L.DIRECT_LIMIT, inv.n, True),
                                  (None, 1, True)):
            if limit is not None:
                L.llama_set_direct_max(s.ctx, limit)
            sub = inv.subset(np.arange(n))
            out = np.full(n, -7, L.DECISION_DTYPE)
            rc = lib.llama_schedule(s.ctx, n, sub.dag.ctypes.data, sub.op_local.ctypes.data,
                                    sub.start_us.ctypes.data, sub.now_us, out.ctypes.data)
            if decided:
                assert rc == L.OK, L.llama_last_error(s.ctx)
                assert L.llama_last_launch_count(s.ctx) == 2
                exp, _ = oracle.schedule(p, sub)
                assert_same(out, exp, f"{n} invocations, limit {limit}")
            else:
                assert rc == L.ETIMEOUT, (n, limit)
        L.llama_set_wait_limit(s.ctx, L.WAIT_LIMIT_DEFAULT)
        L.llama_set_direct_max(s.ctx, L.DIRECT_DEFAULT)
        # the static entry point, a fifth of the invocations invalid
        sub = inv.subset(np.arange(L.DIRECT_DEFAULT))
        sub.dag[::5] = -1
        exp, rc_o = oracle.schedule(p, sub)
        assert rc_o == oracle.EINVAL
        dev = torch.device("cuda", 0)
        stream = torch.cuda.Stream(device=dev)
        d = [torch.from_numpy(a).to(dev) for a in (sub.dag, sub.op_local, sub.start_us)]
        o = torch.full((sub.n * 24,), 0xA5, dtype=torch.uint8, device=dev)
        sp = ctypes.c_void_p(stream.cuda_stream)
        assert lib.llama_schedule_static(s.ctx, sub.n, d[0].data_ptr(), d[1].data_ptr(), d[2].data_ptr(),
                                         sub.now_us, o.data_ptr(), sp) == L.OK
        n_bad, tmo = ctypes.c_int64(-1), ctypes.c_int32(-1)
        assert lib.llama_static_status(s.ctx, sp, ctypes.byref(n_bad), ctypes.byref(tmo)) == L.OK
        stream.synchronize()
        assert (n_bad.value, tmo.value) == (int((sub.dag < 0).sum()), 0)
        assert L.llama_last_launch_count(s.ctx) == 2
        assert_same(o.cpu().numpy().view(L.DECISION_DTYPE), exp, "static entry point")
