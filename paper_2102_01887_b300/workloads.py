"""Seeded synthetic inputs shaped like the paper's video pipelines.

This module only draws inputs: DAG shapes, per-operation configuration tables
and pending invocations.  It performs none of the scheduling arithmetic (no
critical path, no slack, no objective), so both the CPU oracle and the CUDA
path can be fed from it without sharing any of the method's code.

Shapes follow the paper's evaluation (Section 6, Table 2): pipelines of a few
operations in sequential, parallel and branching form, per-operation
configuration spaces spanned by knobs (resolution, batch size, sampling rate)
times hardware type and resource size (Section 4.2, Section 5), the reference
configuration being the smallest CPU configuration, one core and batch one
(Section 3.2).  Latencies are int32 microseconds and costs int64 nano-dollars
per invocation, i.e. the C(x)/B(x) term of Eq. 1.  The price of a resource is
per resource-microsecond, as in the paper's cost model (Section 6, "Resource
requests and cost model").

Workloads (seed = workload number - 1):

* ``tiny``    -- 1 DAG decode -> detect -> {face | car}; 8 knobs x 3 hardware
  types = 24 configurations per operation; 64 invocations.
* ``medium``  -- 16 random DAGs of 10-20 operations, 1,024 configurations per
  operation, 65,536 invocations.
* ``batched`` -- 256 random DAGs of 5-60 operations, Zipf(1.2) configuration
  space sizes over 96..8,192, 1,048,576 invocations.
* ``batched_large`` -- 512 DAGs whose operations all have 8,192
  configurations (tables far larger than L2), few invocations per operation.
* ``random_small`` -- tiny random problems with many ties, used by the tests.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

N_HW = 3
INT32_MAX = 2**31 - 1

# (hardware type, resource size) pairs in hardware-major order: CPU-small
# (cores), CPU-large (cores), GPU (GB of device memory).
HW_RES = [(0, 1), (0, 2), (1, 4), (1, 8), (1, 16), (2, 2), (2, 4), (2, 8)]
# Nano-dollars per resource-microsecond for each hardware type.
PRICE = [1.0, 1.1, 3.0]
# Total resources of each backend (cores, cores, GB).
RES_TOTAL = [320, 640, 32]
RESOLUTIONS = [360, 480, 720, 1080]
BATCHES = [1, 2, 4, 8, 16, 32, 64, 128]
N_SAMPLING = 5
ZIPF_SIZES = [96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048, 3072, 4096, 6144, 8192]


@dataclasses.dataclass
class Problem:
    """Pipelines plus per-operation configuration tables (SoA, flat)."""

    n_hw: int
    dag_op_off: np.ndarray  # int32[n_dags+1]: global op ids of DAG d are [off[d], off[d+1])
    row_ptr: np.ndarray  # int32[n_ops+1]: CSR over global op ids (successors)
    col: np.ndarray  # int32[n_edges]: successor global op ids
    slo_us: np.ndarray  # int64[n_dags]: end-to-end latency target per DAG
    cfg_off: np.ndarray  # int64[n_ops+1]: configs of op v are [cfg_off[v], cfg_off[v+1])
    hw_off: np.ndarray  # int32[n_ops*(n_hw+1)]: op-local start of each hardware segment
    lat_us: np.ndarray  # int32[n_cfg]
    cost_nd: np.ndarray  # int64[n_cfg]: cost per invocation, C(x)/B(x)
    ref_cfg: np.ndarray  # int32[n_ops]: op-local reference configuration
    batch: Optional[np.ndarray] = None  # int32[n_cfg]
    res: Optional[np.ndarray] = None  # int32[n_cfg]
    res_total: Optional[np.ndarray] = None  # int32[n_hw]
    q_us: Optional[np.ndarray] = None  # int64[n_hw]: queueing time per backend
    knobs: Optional["Knobs"] = None  # knob values behind every configuration

    @property
    def n_dags(self) -> int:
        return int(self.dag_op_off.shape[0] - 1)

    @property
    def n_ops(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def n_cfg(self) -> int:
        return int(self.lat_us.shape[0])

    def table_bytes(self) -> int:
        """Bytes of the latency + cost columns (12 B per configuration)."""
        return int(self.lat_us.nbytes + self.cost_nd.nbytes)


@dataclasses.dataclass
class Knobs:
    """Knob values of every configuration and descriptors of every operation
    (what a profiler knows about a configuration besides its latency)."""

    hw: np.ndarray  # int8[n_cfg]: hardware type
    res_idx: np.ndarray  # int8[n_cfg]: processing resolution, index into RESOLUTIONS
    samp_idx: np.ndarray  # int8[n_cfg]: sampling rate index
    variant: np.ndarray  # float32[n_cfg]: variant speed factor
    op_base_us: np.ndarray  # float64[n_ops]: the operation's base latency
    op_gpu_speed: np.ndarray  # float64[n_ops]


@dataclasses.dataclass
class Invocations:
    """Pending invocations (SoA) and the scheduling instant."""

    dag: np.ndarray  # int32[n]
    op_local: np.ndarray  # int32[n]
    start_us: np.ndarray  # int64[n]: start time of the invocation's pipeline instance
    now_us: int

    @property
    def n(self) -> int:
        return int(self.dag.shape[0])

    def subset(self, idx: np.ndarray) -> "Invocations":
        return Invocations(self.dag[idx], self.op_local[idx], self.start_us[idx], self.now_us)


# ----------------------------------------------------------------------------
# DAG shapes
# ----------------------------------------------------------------------------

def _random_dag_edges(rng: np.random.Generator, n: int, p_branch: float = 0.2,
                      fan_max: int = 4, p_sink: float = 0.1) -> list[list[int]]:
    """Local successor lists of a random DAG on ops 0..n-1 (topologically numbered).

    An operation is a branch with probability ``p_branch`` (fan-out 2..fan_max,
    the conditional-flow pattern of Fig. 1), otherwise it has one successor, or
    none with probability ``p_sink``.  Every operation other than 0 is given a
    predecessor so that operation 0 is the single input operation.
    """
    succ: list[set[int]] = [set() for _ in range(n)]
    for v in range(n - 1):
        later = n - 1 - v
        if rng.random() < p_branch:
            fan = int(rng.integers(2, fan_max + 1))
        elif v > 0 and rng.random() < p_sink:
            fan = 0
        else:
            fan = 1
        fan = min(fan, later)
        if fan:
            succ[v].update(int(w) for w in rng.choice(np.arange(v + 1, n), size=fan, replace=False))
    has_pred = np.zeros(n, dtype=bool)
    for v in range(n):
        for w in succ[v]:
            has_pred[w] = True
    for v in range(1, n):
        if not has_pred[v]:
            succ[int(rng.integers(0, v))].add(v)
    return [sorted(s) for s in succ]


def _csr(dags: list[list[list[int]]]) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Concatenate local successor lists into global-id CSR arrays."""
    dag_op_off = [0]
    row_ptr = [0]
    col: list[int] = []
    for succ in dags:
        base = dag_op_off[-1]
        for s in succ:
            col.extend(base + w for w in s)
            row_ptr.append(len(col))
        dag_op_off.append(base + len(succ))
    return (np.asarray(dag_op_off, dtype=np.int32), np.asarray(row_ptr, dtype=np.int32),
            np.asarray(col, dtype=np.int32))


# ----------------------------------------------------------------------------
# Configuration tables
# ----------------------------------------------------------------------------

def _speed(h: np.ndarray, r: np.ndarray, gpu_speed: float) -> np.ndarray:
    s = np.where(h == 0, r.astype(np.float64) ** 0.9, 1.15 * r.astype(np.float64) ** 0.85)
    return np.where(h == 2, gpu_speed * (r.astype(np.float64) / 2.0) ** 0.35, s)


def _knob_table(rng: np.random.Generator, n: int, base: float, gpu_speed: float):
    """One operation's table of ``n`` configurations, hardware-major.

    The full knob grid is (hardware, resource) x variant x resolution x batch
    x sampling rate; it is trimmed by a seeded removal down to ``n`` entries,
    never removing the reference configuration (CPU-small, 1 core, variant 0,
    full resolution, batch 1, first sampling rate).  Sampling rate has no
    latency effect, which deliberately creates ties.
    """
    n_var = max(1, math.ceil(n / (len(HW_RES) * len(RESOLUTIONS) * len(BATCHES) * N_SAMPLING)))
    var_f = np.concatenate([[1.0], rng.uniform(0.3, 3.0, n_var - 1)])
    hr, va, re, ba, sa = np.meshgrid(np.arange(len(HW_RES)), np.arange(n_var),
                                     np.arange(len(RESOLUTIONS)), np.arange(len(BATCHES)),
                                     np.arange(N_SAMPLING), indexing="ij")
    hr, va, re, ba = hr.ravel(), va.ravel(), re.ravel(), ba.ravel()
    total = hr.shape[0]
    ref_full = int(np.flatnonzero((hr == 0) & (va == 0) & (re == len(RESOLUTIONS) - 1)
                                  & (ba == 0) & (sa.ravel() == 0))[0])
    others = np.delete(np.arange(total), ref_full)
    keep = np.sort(np.concatenate([[ref_full], rng.choice(others, size=n - 1, replace=False)]))
    hr, va, re, ba = hr[keep], va[keep], re[keep], ba[keep]
    h = np.asarray([HW_RES[i][0] for i in range(len(HW_RES))])[hr]
    r = np.asarray([HW_RES[i][1] for i in range(len(HW_RES))])[hr]
    res_f = (np.asarray(RESOLUTIONS, dtype=np.float64)[re] / 1080.0) ** 1.5
    b = np.asarray(BATCHES)[ba]
    lat = np.rint(base * var_f[va] * res_f * b.astype(np.float64) ** 0.8 / _speed(h, r, gpu_speed))
    lat = lat + rng.integers(0, 1000, size=n)
    lat = np.clip(lat, 1, INT32_MAX - 1).astype(np.int64)
    price = np.asarray(PRICE)[h]
    cost = np.rint(lat.astype(np.float64) * r * price / b).astype(np.int64)
    hw_off = np.searchsorted(h, np.arange(N_HW + 1), side="left").astype(np.int32)
    ref = int(np.searchsorted(keep, ref_full))
    knobs = (h.astype(np.int8), re.astype(np.int8), sa.ravel()[keep].astype(np.int8),
             var_f[va].astype(np.float32))
    return lat.astype(np.int32), cost, b.astype(np.int32), r.astype(np.int32), hw_off, ref, knobs


def _assemble(rng: np.random.Generator, dags: list[list[list[int]]], sizes: np.ndarray,
              slo_fn, knobs: bool = True, q_max: int = 0) -> Problem:
    dag_op_off, row_ptr, col = _csr(dags)
    n_ops = int(dag_op_off[-1])
    lats, costs, batches, ress, hw_offs, refs, kn, bases, speeds = [], [], [], [], [], [], [], [], []
    for v in range(n_ops):
        base = math.exp(rng.uniform(math.log(5_000.0), math.log(2_000_000.0)))
        gpu_speed = rng.uniform(2.0, 12.0)
        lat, cost, b, r, hw_off, ref, k = _knob_table(rng, int(sizes[v]), base, gpu_speed)
        lats.append(lat), costs.append(cost), hw_offs.append(hw_off), refs.append(ref)
        kn.append(k), bases.append(base), speeds.append(gpu_speed)
        if knobs:
            batches.append(b), ress.append(r)
    cfg_off = np.zeros(n_ops + 1, dtype=np.int64)
    cfg_off[1:] = np.cumsum(sizes)
    lat_us = np.concatenate(lats)
    ref_cfg = np.asarray(refs, dtype=np.int32)
    ref_lat = lat_us[cfg_off[:-1] + ref_cfg]
    slo = slo_fn(dag_op_off, ref_lat)
    q = rng.integers(0, q_max + 1, size=N_HW).astype(np.int64) if q_max else np.zeros(N_HW, np.int64)
    return Problem(
        n_hw=N_HW, dag_op_off=dag_op_off, row_ptr=row_ptr, col=col,
        slo_us=np.clip(slo, 1, INT32_MAX).astype(np.int64), cfg_off=cfg_off,
        hw_off=np.concatenate(hw_offs).astype(np.int32), lat_us=lat_us,
        cost_nd=np.concatenate(costs).astype(np.int64), ref_cfg=ref_cfg,
        batch=np.concatenate(batches) if knobs else None,
        res=np.concatenate(ress) if knobs else None,
        res_total=np.asarray(RES_TOTAL, dtype=np.int32), q_us=q,
        knobs=Knobs(*(np.concatenate([k[j] for k in kn]) for j in range(4)),
                    op_base_us=np.asarray(bases), op_gpu_speed=np.asarray(speeds)))


def _invocations(rng: np.random.Generator, p: Problem, n_inv: int, now_us: int) -> Invocations:
    """Invocations with operations uniform over all ops, elapsed time uniform in [0, SLO)."""
    gop = rng.integers(0, p.n_ops, size=n_inv)
    dag = (np.searchsorted(p.dag_op_off, gop, side="right") - 1).astype(np.int32)
    op_local = (gop - p.dag_op_off[dag]).astype(np.int32)
    elapsed = (rng.random(n_inv) * p.slo_us[dag]).astype(np.int64)
    return Invocations(dag, op_local, (now_us - elapsed).astype(np.int64), now_us)


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------

def tiny(seed: int = 0) -> tuple[Problem, Invocations]:
    """AMBER-Alert-like DAG: 0 decode -> 1 detect -> {2 face-match | 3 car-match}.

    Latency = base (log-uniform 5 ms..2 s) x knob factor (uniform 0.3..3.0) /
    hardware speedup {1, 2.5, 6}; cost = latency x price {1, 4, 9} nano-$/us;
    configuration index = hw * 8 + knob; 64 invocations, elapsed uniform in
    [0, 5 s), SLO 5 s, no queueing.
    """
    rng = np.random.default_rng(seed)
    n_ops, n_knob = 4, 8
    speed = np.asarray([1.0, 2.5, 6.0])
    price = np.asarray([1, 4, 9], dtype=np.int64)
    base = np.exp(rng.uniform(math.log(5_000.0), math.log(2_000_000.0), n_ops))
    knob = rng.uniform(0.3, 3.0, (n_ops, n_knob))
    lat = np.maximum(1, np.rint(base[:, None, None] * knob[:, None, :] / speed[None, :, None]))
    lat = lat.astype(np.int64).reshape(n_ops, N_HW * n_knob)
    cost = lat * np.repeat(price, n_knob)[None, :]
    dag_op_off, row_ptr, col = _csr([[[1], [2, 3], [], []]])
    p = Problem(
        n_hw=N_HW, dag_op_off=dag_op_off, row_ptr=row_ptr, col=col,
        slo_us=np.asarray([5_000_000], dtype=np.int64),
        cfg_off=np.arange(0, (n_ops + 1) * 24, 24, dtype=np.int64),
        hw_off=np.tile(np.asarray([0, 8, 16, 24], dtype=np.int32), n_ops),
        lat_us=lat.ravel().astype(np.int32), cost_nd=cost.ravel(),
        ref_cfg=np.zeros(n_ops, dtype=np.int32),
        batch=np.ones(n_ops * 24, dtype=np.int32), res=np.ones(n_ops * 24, dtype=np.int32),
        res_total=np.asarray([1, 1, 1], dtype=np.int32), q_us=np.zeros(N_HW, dtype=np.int64))
    now = 10**7
    op = rng.integers(0, n_ops, 64)
    elapsed = rng.integers(0, 5_000_000, 64)
    inv = Invocations(np.zeros(64, np.int32), op.astype(np.int32), (now - elapsed).astype(np.int64), now)
    return p, inv


def medium(seed: int = 1, n_inv: int = 65_536, inv_seed: Optional[int] = None) -> tuple[Problem, Invocations]:
    """16 random DAGs of 10-20 ops, 1,024 configurations per op, 65,536 invocations.

    SLO of a DAG = U(0.5, 2) x half the sum of its operations' reference
    latencies (a generator-side scale, not the critical path).
    """
    rng = np.random.default_rng(seed)
    dags = [_random_dag_edges(rng, int(rng.integers(10, 21))) for _ in range(16)]
    n_ops = sum(len(d) for d in dags)

    def slo_fn(off, ref_lat):
        sums = np.add.reduceat(ref_lat.astype(np.float64), off[:-1])
        return np.rint(rng.uniform(0.5, 2.0, off.shape[0] - 1) * 0.5 * sums)

    p = _assemble(rng, dags, np.full(n_ops, 1024), slo_fn, q_max=100_000)
    inv_rng = rng if inv_seed is None else np.random.default_rng(inv_seed)
    return p, _invocations(inv_rng, p, n_inv, 10**11)


def _zipf_sizes(rng: np.random.Generator, n: int, s: float = 1.2) -> np.ndarray:
    w = np.arange(1, len(ZIPF_SIZES) + 1, dtype=np.float64) ** -s
    return np.asarray(ZIPF_SIZES)[rng.choice(len(ZIPF_SIZES), size=n, p=w / w.sum())]


def _log_uniform_slo(rng: np.random.Generator):
    def slo_fn(off, ref_lat):
        return np.rint(np.exp(rng.uniform(math.log(0.5e6), math.log(60e6), off.shape[0] - 1)))
    return slo_fn


def batched(seed: int = 2, n_inv: int = 1_048_576, n_dags: int = 256,
            inv_seed: Optional[int] = None) -> tuple[Problem, Invocations]:
    """256 DAGs of 5-60 ops, Zipf(1.2) config-space sizes 96..8,192, SLO log-uniform 0.5-60 s."""
    rng = np.random.default_rng(seed)
    dags = [_random_dag_edges(rng, int(rng.integers(5, 61))) for _ in range(n_dags)]
    n_ops = sum(len(d) for d in dags)
    p = _assemble(rng, dags, _zipf_sizes(rng, n_ops), _log_uniform_slo(rng), q_max=100_000)
    inv_rng = rng if inv_seed is None else np.random.default_rng(inv_seed)
    return p, _invocations(inv_rng, p, n_inv, 10**11)


def batched_large(seed: int = 3, n_inv: int = 32_768, n_dags: int = 512,
                  inv_seed: Optional[int] = None) -> tuple[Problem, Invocations]:
    """512 DAGs of 5-60 ops, every op with 8,192 configurations (tables >> L2).

    Few invocations per operation, so each table is streamed from HBM about
    once per call.
    """
    rng = np.random.default_rng(seed)
    dags = [_random_dag_edges(rng, int(rng.integers(5, 61))) for _ in range(n_dags)]
    n_ops = sum(len(d) for d in dags)
    p = _assemble(rng, dags, np.full(n_ops, 8192), _log_uniform_slo(rng), q_max=100_000)
    inv_rng = rng if inv_seed is None else np.random.default_rng(inv_seed)
    return p, _invocations(inv_rng, p, n_inv, 10**11)


def dag_sizes(seed: int = 4, sizes: tuple = (1, 3, 40, 100, 126, 127, 200, 511, 513, 1500, 12),
              n_cfg: int = 24, n_inv: int = 16_384) -> tuple[Problem, Invocations]:
    """DAGs of the given op counts side by side (small to 1,500 ops), small tables.

    Shapes from tens to thousands of operations in one problem, with SLOs
    log-uniform 0.5-60 s.
    """
    rng = np.random.default_rng(seed)
    dags = [_random_dag_edges(rng, int(n)) for n in sizes]
    n_ops = sum(len(d) for d in dags)
    p = _assemble(rng, dags, np.full(n_ops, n_cfg), _log_uniform_slo(rng), q_max=100_000)
    return p, _invocations(rng, p, n_inv, 10**11)


def random_small(seed: int, max_dags: int = 3, max_ops: int = 6, max_cfg: int = 8,
                 n_inv: int = 64, value_range: int = 40) -> tuple[Problem, Invocations]:
    """Tiny random problems with small value ranges, so ties and boundary hits are common.

    Latencies and costs are drawn from 1..value_range; SLOs from a similar
    range; elapsed times sometimes exceed the SLO and queueing times are
    sometimes nonzero, so clamped (R <= 0) slack occurs as well.
    """
    rng = np.random.default_rng(seed)
    nd = int(rng.integers(1, max_dags + 1))
    dags = [_random_dag_edges(rng, int(rng.integers(1, max_ops + 1)), p_branch=0.4, p_sink=0.2)
            for _ in range(nd)]
    dag_op_off, row_ptr, col = _csr(dags)
    n_ops = int(dag_op_off[-1])
    sizes = rng.integers(1, max_cfg + 1, size=n_ops)
    cfg_off = np.zeros(n_ops + 1, dtype=np.int64)
    cfg_off[1:] = np.cumsum(sizes)
    n_cfg = int(cfg_off[-1])
    hw_off = []
    for n in sizes:
        cuts = np.sort(rng.integers(0, n + 1, size=N_HW - 1))
        hw_off.append(np.concatenate([[0], cuts, [n]]))
    p = Problem(
        n_hw=N_HW, dag_op_off=dag_op_off, row_ptr=row_ptr, col=col,
        slo_us=rng.integers(1, value_range * 6, size=nd).astype(np.int64), cfg_off=cfg_off,
        hw_off=np.concatenate(hw_off).astype(np.int32),
        lat_us=rng.integers(1, value_range + 1, size=n_cfg).astype(np.int32),
        cost_nd=rng.integers(0, value_range + 1, size=n_cfg).astype(np.int64),
        ref_cfg=np.asarray([rng.integers(0, n) for n in sizes], dtype=np.int32),
        batch=rng.integers(1, 5, size=n_cfg).astype(np.int32),
        res=rng.integers(1, 5, size=n_cfg).astype(np.int32),
        res_total=rng.integers(1, 9, size=N_HW).astype(np.int32),
        q_us=(rng.integers(0, value_range, size=N_HW) * (rng.random(N_HW) < 0.5)).astype(np.int64))
    now = 10**6
    gop = rng.integers(0, n_ops, size=n_inv)
    dag = (np.searchsorted(dag_op_off, gop, side="right") - 1).astype(np.int32)
    elapsed = rng.integers(0, value_range * 8, size=n_inv)
    inv = Invocations(dag, (gop - dag_op_off[dag]).astype(np.int32), (now - elapsed).astype(np.int64), now)
    return p, inv


WORKLOADS = {"tiny": tiny, "medium": medium, "batched": batched, "batched_large": batched_large}


# ----------------------------------------------------------------------------
# Content-dependent latency: the world the learned surrogate is trained on
# ----------------------------------------------------------------------------
#
# The profile table holds each configuration's latency measured on reference
# content.  Real invocations carry frames whose content changes the latency
# (the paper's Fig. 3 motivates this: the same operation on different videos).
# Here an operation has one of N_OP_TYPES kinds, and its latency on content c
# is the profiled latency times exp(log_factor(kind, knobs, c) + noise), the
# factor being 0 on the reference content.  Branch fan-out grows with the
# number of objects for the branching kinds.

N_OP_TYPES = 8
N_BRANCH_TYPES = 2  # kinds 0 and 1 fan out per detected object
N_CFG_FEATURES = 32
N_CONTENT_FEATURES = 16
N_FEATURES = N_CFG_FEATURES + N_CONTENT_FEATURES
REF_OBJECTS, REF_MOTION, REF_IN_RES = 10, 0.5, len(RESOLUTIONS) - 1
LATENCY_NOISE_SIGMA = 0.1


@dataclasses.dataclass
class ContentWorld:
    """Per-operation kinds and the per-kind sensitivities of latency to content."""

    op_type: np.ndarray  # int8[n_ops]
    a_obj: np.ndarray  # float64[N_OP_TYPES]: per 25 objects above the reference
    b_motion: np.ndarray  # per unit of motion above the reference
    s_batch: np.ndarray  # objects x batch interaction (saturating at batch 16)
    r_res: np.ndarray  # per unit of (input resolution / 1080)^1.5 below 1
    f_fan: np.ndarray  # expected extra fan-out per object (branching kinds)


@dataclasses.dataclass
class Content:
    """Frame content of invocations."""

    n_obj: np.ndarray  # int32[n]: objects in the frame
    motion: np.ndarray  # float32[n]: motion score in [0, 1]
    in_res: np.ndarray  # int8[n]: input resolution, index into RESOLUTIONS

    @property
    def n(self) -> int:
        return int(self.n_obj.shape[0])


def content_world(p: Problem, seed: int = 101) -> ContentWorld:
    rng = np.random.default_rng(seed)
    return ContentWorld(op_type=rng.integers(0, N_OP_TYPES, size=p.n_ops).astype(np.int8),
                        a_obj=rng.uniform(0.2, 1.2, N_OP_TYPES), b_motion=rng.uniform(0.0, 0.6, N_OP_TYPES),
                        s_batch=rng.uniform(0.0, 0.5, N_OP_TYPES), r_res=rng.uniform(0.0, 0.8, N_OP_TYPES),
                        f_fan=rng.uniform(0.02, 0.1, N_OP_TYPES))


def draw_content(rng: np.random.Generator, n: int) -> Content:
    """Objects ~ Poisson(lambda), lambda ~ U(0, 50); motion ~ U(0, 1); input resolution uniform."""
    lam = rng.uniform(0.0, 50.0, n)
    return Content(rng.poisson(lam).astype(np.int32), rng.uniform(0.0, 1.0, n).astype(np.float32),
                   rng.integers(0, len(RESOLUTIONS), n).astype(np.int8))


def reference_content(n: int) -> Content:
    return Content(np.full(n, REF_OBJECTS, np.int32), np.full(n, REF_MOTION, np.float32),
                   np.full(n, REF_IN_RES, np.int8))


def config_features(p: Problem, cw: ContentWorld, gop: np.ndarray, cfg: np.ndarray) -> np.ndarray:
    """Features of configurations (global op ids, op-local indices): float32[m, 32]."""
    k = p.knobs
    g = p.cfg_off[gop] + cfg
    m = g.shape[0]
    f = np.zeros((m, N_CFG_FEATURES), np.float32)
    f[np.arange(m), k.hw[g]] = 1.0
    f[:, 3] = np.log2(p.res[g]) / 4.0 if p.res is not None else 0.0
    f[:, 4] = np.log2(p.batch[g]) / 7.0 if p.batch is not None else 0.0
    f[np.arange(m), 5 + k.res_idx[g]] = 1.0
    f[np.arange(m), 9 + k.samp_idx[g]] = 1.0
    f[:, 14] = np.log(k.variant[g])
    f[:, 15] = (np.log(k.op_base_us[gop]) - math.log(5e3)) / math.log(400.0)
    f[:, 16] = k.op_gpu_speed[gop] / 12.0
    f[:, 17] = (np.log(p.lat_us[g]) - 8.0) / 8.0
    f[np.arange(m), 18 + cw.op_type[gop]] = 1.0
    return f


def content_features(c: Content) -> np.ndarray:
    """Features of frame content: float32[n, 16]."""
    f = np.zeros((c.n, N_CONTENT_FEATURES), np.float32)
    f[:, 0] = c.n_obj / 50.0
    f[:, 1] = np.log1p(c.n_obj) / 4.0
    f[:, 2] = c.motion
    f[np.arange(c.n), 3 + c.in_res] = 1.0
    f[:, 7] = 1.0
    return f


def true_log_factor(p: Problem, cw: ContentWorld, gop: np.ndarray, cfg: np.ndarray, c: Content) -> np.ndarray:
    """log(latency on content c / profiled latency), without noise (0 on reference content)."""
    t = cw.op_type[gop]
    b = p.batch[p.cfg_off[gop] + cfg].astype(np.float64)
    dobj = c.n_obj.astype(np.float64) - REF_OBJECTS
    res = (np.asarray(RESOLUTIONS, np.float64)[c.in_res] / 1080.0) ** 1.5
    return (cw.a_obj[t] * dobj / 25.0 + cw.b_motion[t] * (c.motion.astype(np.float64) - REF_MOTION)
            + cw.s_batch[t] * np.minimum(b, 16.0) / 16.0 * dobj / 50.0 + cw.r_res[t] * (res - 1.0))


def expected_fanout(cw: ContentWorld, gop: np.ndarray, c: Content) -> np.ndarray:
    t = cw.op_type[gop]
    return 1.0 + np.where(t < N_BRANCH_TYPES, cw.f_fan[t] * c.n_obj, 0.0)


def surrogate_training_set(p: Problem, cw: ContentWorld, n: int, seed: int = 202):
    """n profiled samples: features float32[n, 48]; targets float32[n, 2] =
    (log latency factor with lognormal noise, sampled fan-out)."""
    rng = np.random.default_rng(seed)
    gop = rng.integers(0, p.n_ops, n)
    cfg = (rng.random(n) * np.diff(p.cfg_off)[gop]).astype(np.int64)
    c = draw_content(rng, n)
    x = np.concatenate([config_features(p, cw, gop, cfg), content_features(c)], axis=1)
    t = np.empty((n, 2), np.float32)
    t[:, 0] = true_log_factor(p, cw, gop, cfg, c) + rng.normal(0.0, LATENCY_NOISE_SIGMA, n)
    t[:, 1] = 1.0 + np.where(cw.op_type[gop] < N_BRANCH_TYPES,
                             rng.poisson(cw.f_fan[cw.op_type[gop]] * c.n_obj), 0)
    return x, t


def invocation_content(seed: int, n: int, reference: bool = False) -> Content:
    """Content of n pending invocations (reference content for all if asked)."""
    return reference_content(n) if reference else draw_content(np.random.default_rng(seed), n)


def latency_noise(seed: int, shape) -> np.ndarray:
    """The lognormal noise of the latencies actually observed (per invocation and configuration)."""
    return np.random.default_rng(seed).normal(0.0, LATENCY_NOISE_SIGMA, shape)
