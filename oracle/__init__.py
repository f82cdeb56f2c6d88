"""ctypes wrapper of the CPU oracle (``llama_oracle.c``).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It never serves the
product path and shares no code with the CUDA library.

The oracle computes, in plain single-threaded C with 128-bit intermediates:
  * the slack of an invocation for each backend, Algorithm 1 (Section 4.1),
    either by enumerating every source-to-sink path (``method="paths"``) or
    through the longest remaining path (``method="critical_path"``);
  * the chosen configuration, by scoring every configuration with Eq. 1
    (Section 4.2) and keeping the best one by plain comparisons.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "llama_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODE_COST_FIRST = 0
MODE_ALPHA = 1
FLAG_FEASIBLE = 1
FLAG_INVALID = 2
OK, EINVAL, ENOMEM, ETOOBIG = 0, -1, -2, -6

DECISION_DTYPE = np.dtype([("cfg", "<i4"), ("lat", "<i4"), ("cost", "<i8"),
                           ("slack", "<i4"), ("flags", "<i4")])


def build(force: bool = False, src: str = _SRC, out: str = _LIB, extra_flags: tuple = ()) -> str:
    """Compile the oracle with gcc into a shared library (plain -O2)."""
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        subprocess.run(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-Wall", "-Werror",
                        *extra_flags, "-o", out, src], check=True)
    return out


class _Problem(ctypes.Structure):
    _fields_ = [
        ("n_dags", ctypes.c_int32), ("n_ops", ctypes.c_int32), ("n_hw", ctypes.c_int32),
        ("mode", ctypes.c_int32),
        ("dag_op_off", ctypes.c_void_p), ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p),
        ("slo_us", ctypes.c_void_p), ("cfg_off", ctypes.c_void_p), ("hw_off", ctypes.c_void_p),
        ("lat_us", ctypes.c_void_p), ("cost_nd", ctypes.c_void_p), ("ref_cfg", ctypes.c_void_p),
        ("batch", ctypes.c_void_p), ("res", ctypes.c_void_p), ("res_total", ctypes.c_void_p),
        ("q_us", ctypes.c_void_p), ("alpha_num", ctypes.c_int64), ("alpha_den", ctypes.c_int64),
    ]


def _bind(lib: ctypes.CDLL) -> ctypes.CDLL:
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.or_topo_order.argtypes = [i32, vp, vp, vp]
    lib.or_critical_path.argtypes = [i32, vp, vp, vp, vp]
    lib.or_slack_from_cp.argtypes = [i64, i64, i64]
    lib.or_slack_from_cp.restype = i64
    lib.or_slack_paths.argtypes = [i32, i32, vp, vp, vp, i32, i64, i64, vp, vp]
    lib.or_select.argtypes = [vp, i32, vp, vp]
    lib.or_slacks.argtypes = [vp, i64, vp, vp, vp, i64, i32, vp]
    lib.or_schedule.argtypes = [vp, i64, vp, vp, vp, i64, i32, vp]
    for f in (lib.or_topo_order, lib.or_critical_path, lib.or_slack_paths, lib.or_select,
              lib.or_slacks, lib.or_schedule):
        f.restype = ctypes.c_int
    return lib


def load(path: str | None = None) -> ctypes.CDLL:
    """Load the oracle library (building it if needed); ``path`` loads another build."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class _Marshalled:
    """Keeps contiguous copies alive while the C struct points at them."""

    def __init__(self, p, mode: int, alpha: tuple[int, int]):
        c = lambda a, dt: None if a is None else np.ascontiguousarray(a, dtype=dt)
        self.arrays = dict(
            dag_op_off=c(p.dag_op_off, np.int32), row_ptr=c(p.row_ptr, np.int32),
            col=c(p.col, np.int32) if p.col.size else np.zeros(1, np.int32),
            slo_us=c(p.slo_us, np.int64), cfg_off=c(p.cfg_off, np.int64),
            hw_off=c(p.hw_off, np.int32), lat_us=c(p.lat_us, np.int32),
            cost_nd=c(p.cost_nd, np.int64), ref_cfg=c(p.ref_cfg, np.int32),
            batch=c(p.batch, np.int32), res=c(p.res, np.int32),
            res_total=c(p.res_total, np.int32),
            q_us=c(p.q_us if p.q_us is not None else np.zeros(p.n_hw, np.int64), np.int64))
        a = self.arrays
        self.struct = _Problem(
            p.n_dags, p.n_ops, p.n_hw, mode,
            *[_ptr(a[k]) for k in ("dag_op_off", "row_ptr", "col", "slo_us", "cfg_off", "hw_off",
                                   "lat_us", "cost_nd", "ref_cfg", "batch", "res", "res_total",
                                   "q_us")],
            int(alpha[0]), int(alpha[1]))


def reference_latency(p) -> np.ndarray:
    """ref[v] = L(reference configuration of v), Section 3.2."""
    return p.lat_us[p.cfg_off[:-1] + p.ref_cfg].astype(np.int64)


def critical_path(p, lib: ctypes.CDLL | None = None) -> np.ndarray:
    lib = lib or load()
    ref = reference_latency(p)
    cp = np.zeros(p.n_ops, dtype=np.int64)
    rp = np.ascontiguousarray(p.row_ptr, np.int32)
    col = np.ascontiguousarray(p.col, np.int32) if p.col.size else np.zeros(1, np.int32)
    rc = lib.or_critical_path(p.n_ops, _ptr(rp), _ptr(col), _ptr(ref), _ptr(cp))
    if rc != OK:
        raise ValueError(f"oracle critical path failed: {rc}")
    return cp


def slack_paths(p, op: int, R: int, max_paths: int = 1_000_000, lib=None) -> tuple[int, int]:
    """Algorithm 1 by path enumeration for global op id ``op``: (slack, number of paths)."""
    lib = lib or load()
    d = int(np.searchsorted(p.dag_op_off, op, side="right") - 1)
    ref = reference_latency(p)
    rp = np.ascontiguousarray(p.row_ptr, np.int32)
    col = np.ascontiguousarray(p.col, np.int32) if p.col.size else np.zeros(1, np.int32)
    s, n = ctypes.c_int64(), ctypes.c_int64()
    rc = lib.or_slack_paths(int(p.dag_op_off[d]), int(p.dag_op_off[d + 1]), _ptr(rp), _ptr(col),
                            _ptr(ref), op, R, max_paths, ctypes.byref(s), ctypes.byref(n))
    if rc != OK:
        raise ValueError(f"oracle path slack failed: {rc}")
    return s.value, n.value


def slacks(p, inv, method: str = "critical_path", lib=None) -> np.ndarray:
    """int64[n_inv, n_hw] slack per invocation and backend (-1 for invalid invocations)."""
    lib = lib or load()
    m = _Marshalled(p, MODE_COST_FIRST, (1, 1))
    out = np.zeros((inv.n, p.n_hw), dtype=np.int64)
    dag = np.ascontiguousarray(inv.dag, np.int32)
    opl = np.ascontiguousarray(inv.op_local, np.int32)
    st = np.ascontiguousarray(inv.start_us, np.int64)
    rc = lib.or_slacks(ctypes.byref(m.struct), inv.n, _ptr(dag), _ptr(opl), _ptr(st),
                       int(inv.now_us), 1 if method == "paths" else 0, _ptr(out))
    if rc != OK:
        raise ValueError(f"oracle slacks failed: {rc}")
    return out


def schedule(p, inv, mode: int = MODE_COST_FIRST, alpha: tuple[int, int] = (1, 1),
             method: str = "critical_path", lib=None) -> tuple[np.ndarray, int]:
    """Decisions (structured array, DECISION_DTYPE) and the oracle's status code."""
    lib = lib or load()
    m = _Marshalled(p, mode, alpha)
    out = np.zeros(inv.n, dtype=DECISION_DTYPE)
    dag = np.ascontiguousarray(inv.dag, np.int32)
    opl = np.ascontiguousarray(inv.op_local, np.int32)
    st = np.ascontiguousarray(inv.start_us, np.int64)
    rc = lib.or_schedule(ctypes.byref(m.struct), inv.n, _ptr(dag), _ptr(opl), _ptr(st),
                         int(inv.now_us), 1 if method == "paths" else 0, _ptr(out))
    if rc not in (OK, EINVAL):
        raise ValueError(f"oracle schedule failed: {rc}")
    return out, rc


def queue_time(p, inv, decisions) -> np.ndarray:
    """Eq. 2 (Section 4.3): per backend, the floor of the sum over the decided
    invocations on it of L(x_i) R(x_i) / R_total(backend), summed exactly in
    integers before one floor division.  Invalid decisions are skipped."""
    H = p.n_hw
    hw = p.hw_off.reshape(p.n_ops, H + 1)
    total = [0] * H
    for i in range(inv.n):
        d = decisions[i]
        if d["cfg"] < 0 or d["flags"] & FLAG_INVALID:
            continue
        v = int(p.dag_op_off[inv.dag[i]]) + int(inv.op_local[i])
        x = int(d["cfg"])
        lam = max(h for h in range(H) if x >= hw[v, h])  # the segment holding x
        total[lam] += int(d["lat"]) * int(p.res[int(p.cfg_off[v]) + x])
    return np.asarray([min(total[h] // int(p.res_total[h]), 2**31 - 1) for h in range(H)], np.int64)


def feedback(p, op, cfg, lat_obs, cost_obs, beta=(1, 4)):
    """Exponential smoothing of the profile tables by measured invocations
    (Section 3.3), in place and in the given order, in exact integers:
    L <- ((d - b) L + b L_obs + d // 2) // d with beta = b / d, the same for the
    cost; observations outside the tables are skipped (their count is returned)."""
    b, d = int(beta[0]), int(beta[1])
    rejected = 0
    for v, x, lo, co in zip(op, cfg, lat_obs, cost_obs):
        v, x, lo, co = int(v), int(x), int(lo), int(co)
        if not (0 <= v < p.n_ops and 0 <= x < int(p.cfg_off[v + 1] - p.cfg_off[v])) or lo < 1 or co < 0 \
                or lo >= 2**31 - 1 or co >= 2**46:
            rejected += 1
            continue
        g = int(p.cfg_off[v]) + x
        L = ((d - b) * int(p.lat_us[g]) + b * lo + d // 2) // d
        p.lat_us[g] = min(max(L, 1), 2**31 - 2)
        p.cost_nd[g] = ((d - b) * int(p.cost_nd[g]) + b * co + d // 2) // d
    return rejected


def backend_objectives(p, inv, alpha=(1, 1)) -> np.ndarray:
    """Eq. 3's per-backend minima (Section 4.4): for every invocation and backend,
    the least Eq. 1 objective among its op's configurations on that backend
    (C/B if feasible, else C/B + floor(a L R / (b B R_total)), saturating);
    INT64_MAX where the backend has none or the invocation is invalid."""
    H = p.n_hw
    a, b = int(alpha[0]), int(alpha[1])
    imax = 2**63 - 1
    sl = slacks(p, inv)
    hw = p.hw_off.reshape(p.n_ops, H + 1)
    out = np.full((inv.n, H), imax, np.int64)
    for i in range(inv.n):
        if sl[i, 0] < 0:
            continue
        v = int(p.dag_op_off[inv.dag[i]]) + int(inv.op_local[i])
        for h in range(H):
            best = imax
            for x in range(int(hw[v, h]), int(hw[v, h + 1])):
                g = int(p.cfg_off[v]) + x
                L, C = int(p.lat_us[g]), int(p.cost_nd[g])
                if L < sl[i, h]:
                    obj = C
                else:
                    obj = min(C + (a * L * int(p.res[g])) // (b * int(p.batch[g]) * int(p.res_total[h])), imax)
                best = min(best, obj)
            out[i, h] = best
    return out


def commit_order(p, inv, decisions, obj_min):
    """Priority-based commit order (Section 4.4): by the backend of each decision,
    then descending affinity (Eq. 3: least objective elsewhere over least on its
    own backend), then index; invalid decisions last.  Returns (order, affinity)."""
    H = p.n_hw
    hw = p.hw_off.reshape(p.n_ops, H + 1)
    keys, aff = [], np.zeros(inv.n)
    for i in range(inv.n):
        d = decisions[i]
        if d["cfg"] < 0 or d["flags"] & FLAG_INVALID:
            keys.append((H, 0.0, i))
            continue
        v = int(p.dag_op_off[inv.dag[i]]) + int(inv.op_local[i])
        lam = max(h for h in range(H) if int(d["cfg"]) >= hw[v, h])
        own = int(obj_min[i, lam])
        other = min(int(obj_min[i, h]) for h in range(H) if h != lam) if H > 1 else 2**63 - 1
        a = (1.0 if other == 0 else float("inf")) if own == 0 else float(other) / float(own)
        aff[i] = a
        keys.append((lam, -a, i))
    order = [k[2] for k in sorted(keys)]
    return np.asarray(order, np.int32), aff
