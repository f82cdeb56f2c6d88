"""Thin Python binding of ``libllama.so`` (the C ABI in ``include/llama.h``).

Argument marshalling only: every step of the scheduling path runs in the
library's CUDA kernels.  Functions carry the C names.  Host arrays are numpy;
device arrays are torch CUDA tensors (PyTorch supplies device memory and
streams, nothing else).  There is no CPU fallback: loading fails loudly if
the shared library is missing.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libllama.so")
# the -DLLAMA_CHECK build (bounds checks that set bits instead of trapping); a
# process selects it with LLAMA_LIB=check before the first load
CHECK_LIB_PATH = os.path.join(_HERE, "libllama_check.so")

OK, EINVAL, ENOMEM, ECUDA, ENOTREADY, ETIMEOUT = 0, -1, -2, -3, -4, -5
MODE_COST_FIRST, MODE_ALPHA = 0, 1
METHOD_SCAN, METHOD_STAIRCASE = 0, 1
FLAG_FEASIBLE, FLAG_INVALID, FLAG_TIMEOUT = 1, 2, 4
WAIT_LIMIT_DEFAULT = 1 << 20
DIRECT_DEFAULT, DIRECT_LIMIT = 1024, 1 << 20
MAX_HW, MAX_CFG = 8, 8192

DECISION_DTYPE = np.dtype([("cfg", "<i4"), ("lat", "<i4"), ("cost", "<i8"),
                           ("slack", "<i4"), ("flags", "<i4")])
assert DECISION_DTYPE.itemsize == 24

EXPORTS = ("llama_create", "llama_destroy", "llama_set_dags", "llama_set_profiles",
           "llama_set_queue", "llama_schedule", "llama_schedule_async", "llama_schedule_static",
           "llama_set_tuning", "llama_set_count_pass", "llama_set_score_occupancy", "llama_set_dlat_stage", "llama_set_method", "llama_reserve",
           "llama_critical_path", "llama_slack", "llama_set_trace_events", "llama_last_launch_count",
           "llama_last_error", "llama_gemm_bf16", "llama_gemm_error",
           "llama_mlp_create", "llama_mlp_destroy", "llama_mlp_set_params", "llama_mlp_get_params",
           "llama_mlp_forward", "llama_mlp_gradients", "llama_mlp_train_step", "llama_mlp_train_epoch", "llama_mlp_last_error",
           "llama_sg_create", "llama_sg_destroy", "llama_sg_schedule", "llama_sg_last_pairs",
           "llama_sg_predictions", "llama_sg_last_error", "llama_sg_set_margin", "llama_sg_invalidate",
           "llama_ws_create", "llama_ws_destroy", "llama_schedule_ws_async", "llama_ws_status", "llama_ws_set_inputs",
           "llama_server_create", "llama_server_destroy", "llama_server_submit", "llama_server_poll",
           "llama_server_drain", "llama_server_stats_get", "llama_queue_time", "llama_feedback",
           "llama_get_profiles", "llama_backend_objectives", "llama_commit_order",
           "llama_static_status", "llama_set_wait_limit", "llama_set_direct_max", "llama_alu_peak", "llama_count_rate", "llama_stragglers", "llama_set_stats_file",
           "llama_check_build", "llama_check_word",
           "llama_loop_create", "llama_loop_destroy", "llama_loop_submit", "llama_loop_tick", "llama_loop_poll",
           "llama_loop_run_arrivals", "llama_sg_run_arrivals",
           "llama_loop_sync", "llama_loop_state_get", "llama_loop_refresh", "llama_loop_ticks_done",
           "llama_loop_start", "llama_loop_stop")
TRACE_EVENTS = 3
TRACE_PHASES = ("bucket", "score")


class LlamaError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"llama error {code}: {message}")
        self.code = code


class llama_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("n_hw", ctypes.c_int32),
                ("alpha_num", ctypes.c_int64), ("alpha_den", ctypes.c_int64),
                ("device", ctypes.c_int32), ("use_graph", ctypes.c_int32)]


class llama_loop_opts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("ring", ctypes.c_int32), ("results", ctypes.c_int32),
                ("max_admit", ctypes.c_int32), ("cq_cap", ctypes.c_int32 * MAX_HW)]


class llama_loop_state(ctypes.Structure):
    _fields_ = [("ticks", ctypes.c_int64), ("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("committed", ctypes.c_int64), ("dispatched", ctypes.c_int64),
                ("results", ctypes.c_int64), ("results_dropped", ctypes.c_int64), ("free_slots", ctypes.c_int32),
                ("sq_len", ctypes.c_int32 * MAX_HW), ("cq_len", ctypes.c_int32 * MAX_HW),
                ("q_us", ctypes.c_int64 * MAX_HW)]


LOOP_REQUEST_DTYPE = np.dtype([("id", "<i8"), ("dag", "<i4"), ("op_local", "<i4"), ("start_us", "<i8")])
LOOP_RESULT_DTYPE = np.dtype([("id", "<i8"), ("kind", "<i4"), ("tick", "<i4"), ("decision", DECISION_DTYPE),
                              ("backend", "<i4"), ("pad", "<i4")])
assert LOOP_REQUEST_DTYPE.itemsize == 24 and LOOP_RESULT_DTYPE.itemsize == 48
LOOP_SPECULATED, LOOP_COMMITTED, LOOP_REJECTED = 1, 2, 3
LOOP_MAX_ADMIT = LOOP_MAX_COMMIT = 1024

_lib = None
_lock = threading.Lock()


def load(path: str = None) -> ctypes.CDLL:
    """Load the CUDA library (the checked build when LLAMA_LIB=check); raises if
    it has not been built."""
    global _lib
    if path is None:
        path = CHECK_LIB_PATH if os.environ.get("LLAMA_LIB") == "check" else LIB_PATH
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with `python -m paper_2102_01887_b300.build`")
        lib = ctypes.CDLL(path)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        sig = {
            "llama_create": ([ctypes.POINTER(vp), ctypes.POINTER(llama_opts)], ctypes.c_int),
            "llama_destroy": ([vp], None),
            "llama_set_dags": ([vp, i32, vp, vp, vp, vp], ctypes.c_int),
            "llama_set_profiles": ([vp, i32, vp, vp, vp, vp, vp, vp, vp, vp], ctypes.c_int),
            "llama_set_queue": ([vp, vp], ctypes.c_int),
            "llama_schedule": ([vp, i64, vp, vp, vp, i64, vp], ctypes.c_int),
            "llama_schedule_async": ([vp, i64, vp, vp, vp, i64, vp, vp], ctypes.c_int),
            "llama_schedule_static": ([vp, i64, vp, vp, vp, i64, vp, vp], ctypes.c_int),
            "llama_set_tuning": ([vp, i32, i32, i32, i32], ctypes.c_int),
            "llama_set_count_pass": ([vp, i32], ctypes.c_int),
            "llama_set_score_occupancy": ([vp, i32], ctypes.c_int),
            "llama_set_dlat_stage": ([vp, i32], ctypes.c_int),
            "llama_set_method": ([vp, i32], ctypes.c_int),
            "llama_reserve": ([vp, i64], ctypes.c_int),
            "llama_critical_path": ([vp, vp], ctypes.c_int),
            "llama_slack": ([vp, i64, vp, vp, vp, i64, vp], ctypes.c_int),
            "llama_set_trace_events": ([vp, vp, i32], ctypes.c_int),
            "llama_last_launch_count": ([vp], ctypes.c_int),
            "llama_last_error": ([vp], ctypes.c_char_p),
            "llama_gemm_bf16": ([vp, vp, vp, vp, vp, i64, i32, i32, i32, vp], ctypes.c_int),
            "llama_gemm_error": ([i32], ctypes.c_int),
            "llama_mlp_create": ([ctypes.POINTER(vp), i32, i64], ctypes.c_int),
            "llama_mlp_destroy": ([vp], None),
            "llama_mlp_set_params": ([vp, vp], ctypes.c_int),
            "llama_mlp_get_params": ([vp, vp], ctypes.c_int),
            "llama_mlp_forward": ([vp, vp, i64, vp, vp], ctypes.c_int),
            "llama_mlp_gradients": ([vp, vp, vp, i64, ctypes.c_float, vp, vp, vp], ctypes.c_int),
            "llama_mlp_train_step": ([vp, vp, vp, i64, ctypes.c_float, ctypes.c_float, vp, vp], ctypes.c_int),
            "llama_mlp_train_epoch": ([vp, vp, vp, i64, vp, i64, i64, ctypes.c_float, ctypes.c_float, vp, vp],
                                      ctypes.c_int),
            "llama_mlp_last_error": ([vp], ctypes.c_char_p),
            "llama_sg_create": ([ctypes.POINTER(vp), vp, vp, i64, i64], ctypes.c_int),
            "llama_sg_destroy": ([vp], None),
            "llama_sg_schedule": ([vp, vp, vp, i64, vp, vp, vp, i64, vp, vp], ctypes.c_int),
            "llama_sg_last_pairs": ([vp], i64),
            "llama_sg_predictions": ([vp, vp, vp, vp, i64, vp], ctypes.c_int),
            "llama_sg_last_error": ([vp], ctypes.c_char_p),
            "llama_sg_set_margin": ([vp, ctypes.c_float], ctypes.c_int),
            "llama_sg_invalidate": ([vp], ctypes.c_int),
            "llama_ws_create": ([vp, i64, ctypes.POINTER(vp)], ctypes.c_int),
            "llama_ws_destroy": ([vp], None),
            "llama_schedule_ws_async": ([vp, vp, i64, vp, vp, vp, i64, vp, vp], ctypes.c_int),
            "llama_ws_set_inputs": ([vp, ctypes.c_int32], ctypes.c_int),
            "llama_ws_status": ([vp, vp, vp], ctypes.c_int),
            "llama_server_create": ([vp, vp, ctypes.POINTER(vp)], ctypes.c_int),
            "llama_server_destroy": ([vp], None),
            "llama_server_submit": ([vp, vp, i64], ctypes.c_int),
            "llama_server_poll": ([vp, vp, i64, vp], ctypes.c_int),
            "llama_server_drain": ([vp, vp, i64, vp, i64], ctypes.c_int),
            "llama_server_stats_get": ([vp, vp], ctypes.c_int),
            "llama_queue_time": ([vp, i64, vp, vp, vp, vp, i32, vp], ctypes.c_int),
            "llama_feedback": ([vp, i64, vp, vp, vp, vp, i32, i32, vp, vp], ctypes.c_int),
            "llama_get_profiles": ([vp, vp, vp], ctypes.c_int),
            "llama_backend_objectives": ([vp, i64, vp, vp, vp, i64, vp, vp], ctypes.c_int),
            "llama_commit_order": ([vp, i64, vp, vp, vp, vp, vp, vp, vp], ctypes.c_int),
            "llama_static_status": ([vp, vp, vp, vp], ctypes.c_int),
            "llama_set_wait_limit": ([vp, i32], ctypes.c_int),
            "llama_set_direct_max": ([vp, i64], ctypes.c_int),
            "llama_alu_peak": ([i32, i32, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
            "llama_count_rate": ([i32, i64, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
                                 ctypes.c_int),
            "llama_stragglers": ([i64, vp, vp, vp, i64, i32, i32, i64, vp, vp, ctypes.POINTER(i64)], ctypes.c_int),
            "llama_set_stats_file": ([vp, ctypes.c_char_p], ctypes.c_int),
            "llama_check_build": ([], ctypes.c_int),
            "llama_check_word": ([vp, vp, i32], ctypes.c_int),
            "llama_loop_create": ([vp, ctypes.POINTER(llama_loop_opts), ctypes.POINTER(vp)], ctypes.c_int),
            "llama_loop_destroy": ([vp], None),
            "llama_loop_submit": ([vp, vp, i64], ctypes.c_int),
            "llama_loop_tick": ([vp, i64, vp], ctypes.c_int),
            "llama_loop_poll": ([vp, vp, i64, ctypes.POINTER(i64)], ctypes.c_int),
            "llama_loop_run_arrivals": ([vp, vp, vp, i64, i64, i64, vp, vp], ctypes.c_int),
            "llama_sg_run_arrivals": ([vp, vp, vp, vp, vp, vp, i64, vp, i64, i64, vp, vp, vp, vp], ctypes.c_int),
            "llama_loop_sync": ([vp], ctypes.c_int),
            "llama_loop_state_get": ([vp, ctypes.POINTER(llama_loop_state)], ctypes.c_int),
            "llama_loop_refresh": ([vp], ctypes.c_int),
            "llama_loop_ticks_done": ([vp], i64),
            "llama_loop_start": ([vp, i64, i32, vp], ctypes.c_int),
            "llama_loop_stop": ([vp], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def _ptr(a) -> Optional[int]:
    """Address of a numpy array or torch tensor (None for None)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


def _check(ctx, rc: int, allow=(OK,)) -> int:
    if rc not in allow:
        raise LlamaError(rc, llama_last_error(ctx))
    return rc


def llama_last_error(ctx) -> str:
    return load().llama_last_error(ctx).decode()


def llama_create(mode: int = MODE_COST_FIRST, n_hw: int = 3, alpha=(1, 1), device: int = 0,
                 use_graph: bool = False) -> ctypes.c_void_p:
    ctx = ctypes.c_void_p()
    o = llama_opts(mode, n_hw, int(alpha[0]), int(alpha[1]), device, int(bool(use_graph)))
    rc = load().llama_create(ctypes.byref(ctx), ctypes.byref(o))
    if rc != OK:
        raise LlamaError(rc, "llama_create failed")
    return ctx


def llama_destroy(ctx) -> None:
    if ctx:
        load().llama_destroy(ctx)


def _c(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


def llama_set_dags(ctx, dag_op_off, row_ptr, col, slo_us) -> None:
    a = [_c(dag_op_off, np.int32), _c(row_ptr, np.int32), _c(col, np.int32), _c(slo_us, np.int64)]
    if a[2].size == 0:
        a[2] = np.zeros(1, np.int32)
    _check(ctx, load().llama_set_dags(ctx, a[0].shape[0] - 1, *[_ptr(x) for x in a]))


def llama_set_profiles(ctx, cfg_off, hw_off, lat_us, cost_nd, ref_cfg, batch=None, res=None,
                       res_total=None) -> None:
    a = [_c(cfg_off, np.int64), _c(hw_off, np.int32), _c(lat_us, np.int32), _c(cost_nd, np.int64),
         _c(ref_cfg, np.int32), _c(batch, np.int32), _c(res, np.int32), _c(res_total, np.int32)]
    _check(ctx, load().llama_set_profiles(ctx, a[0].shape[0] - 1, *[_ptr(x) for x in a]))


def llama_set_queue(ctx, q_us) -> None:
    q = _c(q_us, np.int64)
    _check(ctx, load().llama_set_queue(ctx, _ptr(q)))


def llama_set_tuning(ctx, lanes_min_vectors: int = 16, inv_per_thread: int = 2,
                     chunk_entries: int = 0, stages: int = 1) -> None:
    _check(ctx, load().llama_set_tuning(ctx, int(lanes_min_vectors), int(inv_per_thread),
                                        int(chunk_entries), int(stages)))


COUNT_PASS_AUTO, COUNT_PASS_ON, COUNT_PASS_OFF = 0, 1, 2


def llama_set_count_pass(ctx, mode: int) -> None:
    _check(ctx, load().llama_set_count_pass(ctx, int(mode)))


def llama_set_score_occupancy(ctx, ctas_per_sm: int) -> None:
    _check(ctx, load().llama_set_score_occupancy(ctx, int(ctas_per_sm)))


DLAT_STAGE_DEFAULT = 4096
WS_INPUTS_IN_PLACE = 0
WS_INPUTS_COPY = 1


def llama_set_dlat_stage(ctx, max_entries: int) -> None:
    _check(ctx, load().llama_set_dlat_stage(ctx, int(max_entries)))


GEMM_RELU = 1


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def llama_gemm_bf16(a, b, bias=None, c_bf16=None, c_f32=None, flags: int = 0, stream=None) -> None:
    """C = A . B^T (+ bias) (ReLU) on the tensor cores; torch CUDA tensors.

    a: [m, k] bf16, b: [n, k] bf16, bias: [n] float32 or None; c_bf16 [m, n]
    bf16 and/or c_f32 [m, n] float32 receive the result.
    """
    m, k = a.shape
    n = b.shape[0]
    ptr = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    rc = load().llama_gemm_bf16(ptr(a), ptr(b), ptr(bias), ptr(c_bf16), ptr(c_f32), m, n, k, int(flags),
                                _stream_ptr(stream))
    if rc != OK:
        raise LlamaError(rc, "gemm_bf16: bad arguments or launch failure")


def llama_gemm_error(clear: bool = True) -> int:
    return load().llama_gemm_error(1 if clear else 0)


MLP_PARAMS = 164672
MLP_INPUTS = 64


class MLP:
    """The latency surrogate's network on one GPU (torch CUDA tensors in and out)."""

    def __init__(self, device: int = 0, max_batch: int = 8192):
        self.h = ctypes.c_void_p()
        rc = load().llama_mlp_create(ctypes.byref(self.h), int(device), int(max_batch))
        if rc != OK:
            raise LlamaError(rc, "mlp_create failed")

    def _check(self, rc):
        if rc != OK:
            raise LlamaError(rc, load().llama_mlp_last_error(self.h).decode())

    def set_params(self, flat) -> None:
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.shape == (MLP_PARAMS,)
        self._check(load().llama_mlp_set_params(self.h, a.ctypes.data))

    def get_params(self) -> np.ndarray:
        a = np.empty(MLP_PARAMS, np.float32)
        self._check(load().llama_mlp_get_params(self.h, a.ctypes.data))
        return a

    def forward(self, x, y, stream=None) -> None:
        self._check(load().llama_mlp_forward(self.h, ctypes.c_void_p(x.data_ptr()), x.shape[0],
                                             ctypes.c_void_p(y.data_ptr()), _stream_ptr(stream)))

    def gradients(self, x, t, w_fan: float, grads=None, loss=None, stream=None) -> None:
        p = lambda v: None if v is None else ctypes.c_void_p(v.data_ptr())
        self._check(load().llama_mlp_gradients(self.h, p(x), p(t), x.shape[0], float(w_fan), p(grads), p(loss),
                                               _stream_ptr(stream)))

    def train_step(self, x, t, w_fan: float, lr: float, loss=None, stream=None) -> None:
        p = lambda v: None if v is None else ctypes.c_void_p(v.data_ptr())
        self._check(load().llama_mlp_train_step(self.h, p(x), p(t), x.shape[0], float(w_fan), float(lr), p(loss),
                                                _stream_ptr(stream)))

    def train_epoch(self, x, t, perm, batch: int, w_fan: float, lr: float, loss_sum=None, stream=None) -> None:
        """Adam steps over the batches perm[b*batch:(b+1)*batch] of x and t
        (perm: int32 device tensor), gathered on the device."""
        p = lambda v: None if v is None else ctypes.c_void_p(v.data_ptr())
        assert perm.dtype.itemsize == 4 and perm.shape[0] % batch == 0
        self._check(load().llama_mlp_train_epoch(self.h, p(x), p(t), x.shape[0], p(perm), perm.shape[0] // batch,
                                                 int(batch), float(w_fan), float(lr), p(loss_sum),
                                                 _stream_ptr(stream)))

    def close(self) -> None:
        if self.h:
            load().llama_mlp_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


EAGAIN = -6
REQUEST_DTYPE = np.dtype([("id", "<i8"), ("dag", "<i4"), ("op_local", "<i4"), ("start_us", "<i8"),
                          ("now_us", "<i8")])
RESULT_DTYPE = np.dtype([("id", "<i8"), ("decision", DECISION_DTYPE), ("submit_ns", "<i8"), ("done_ns", "<i8")])
assert REQUEST_DTYPE.itemsize == 32 and RESULT_DTYPE.itemsize == 48


class llama_server_opts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("max_batch", ctypes.c_int32), ("memory_budget", ctypes.c_int64),
                ("max_queue", ctypes.c_int64)]


class llama_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("refused", ctypes.c_int64),
                ("batches", ctypes.c_int64), ("slots", ctypes.c_int32), ("max_in_flight", ctypes.c_int32),
                ("overlapped", ctypes.c_int64), ("queue_peak", ctypes.c_int64),
                ("device_busy_ms", ctypes.c_double), ("device_span_ms", ctypes.c_double)]


class Server:
    """Continuous-batching serving loop over a context (see include/llama_server.h)."""

    def __init__(self, sched, slots: int = 4, max_batch: int = 4096, memory_budget: int = 0, max_queue: int = 0):
        self.h = ctypes.c_void_p()
        opts = llama_server_opts(slots, max_batch, memory_budget, max_queue)
        rc = load().llama_server_create(sched.ctx, ctypes.byref(opts), ctypes.byref(self.h))
        if rc != OK:
            raise LlamaError(rc, "server_create failed")
        self.buf = np.zeros(1 << 16, RESULT_DTYPE)

    def submit(self, req: np.ndarray) -> int:
        req = np.ascontiguousarray(req, REQUEST_DTYPE)
        return load().llama_server_submit(self.h, req.ctypes.data, req.shape[0])

    def poll(self) -> np.ndarray:
        n = ctypes.c_int64()
        rc = load().llama_server_poll(self.h, self.buf.ctypes.data, self.buf.shape[0], ctypes.byref(n))
        if rc != OK:
            raise LlamaError(rc, "server_poll failed")
        return self.buf[:n.value].copy()

    def drain(self, timeout_ms: int = 60000) -> np.ndarray:
        out = []
        while True:
            n = ctypes.c_int64()
            rc = load().llama_server_drain(self.h, self.buf.ctypes.data, self.buf.shape[0], ctypes.byref(n),
                                           int(timeout_ms))
            if rc != OK:
                raise LlamaError(rc, "server_drain failed")
            out.append(self.buf[:n.value].copy())
            if n.value < self.buf.shape[0]:
                return np.concatenate(out)

    def stats(self) -> dict:
        st = llama_server_stats()
        rc = load().llama_server_stats_get(self.h, ctypes.byref(st))
        if rc != OK:
            raise LlamaError(rc, "server_stats failed")
        return {f: getattr(st, f) for f, _ in llama_server_stats._fields_}

    def close(self):
        if self.h:
            load().llama_server_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def llama_queue_time(ctx, dag, op_local, dec, q_out=None, apply: bool = True, stream=None) -> None:
    """Eq. 2 on device tensors: dag, op_local int32 [n], dec uint8 [n*24] (decisions)."""
    v = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    _check(ctx, load().llama_queue_time(ctx, dag.shape[0], v(dag), v(op_local), v(dec), v(q_out),
                                        1 if apply else 0, _stream_ptr(stream)))


def llama_feedback(ctx, op, cfg, lat_us, cost_nd, beta=(1, 4), rejected=None, stream=None) -> None:
    """Exponential-smoothing feedback from device tensors (int32 op, cfg, lat; int64 cost)."""
    v = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    _check(ctx, load().llama_feedback(ctx, op.shape[0], v(op), v(cfg), v(lat_us), v(cost_nd), int(beta[0]),
                                      int(beta[1]), v(rejected), _stream_ptr(stream)))


def llama_backend_objectives(ctx, dag, op_local, start, now_us: int, obj_min, stream=None) -> None:
    v = lambda t: ctypes.c_void_p(t.data_ptr())
    _check(ctx, load().llama_backend_objectives(ctx, dag.shape[0], v(dag), v(op_local), v(start), int(now_us),
                                                v(obj_min), _stream_ptr(stream)))


def llama_commit_order(ctx, dag, op_local, dec, obj_min, order, affinity=None, stream=None) -> None:
    v = lambda t: None if t is None else ctypes.c_void_p(t.data_ptr())
    _check(ctx, load().llama_commit_order(ctx, dag.shape[0], v(dag), v(op_local), v(dec), v(obj_min), v(order),
                                          v(affinity), _stream_ptr(stream)))


def llama_get_profiles(ctx, n_cfg: int):
    lat = np.empty(n_cfg, np.int32)
    cost = np.empty(n_cfg, np.int64)
    _check(ctx, load().llama_get_profiles(ctx, lat.ctypes.data, cost.ctypes.data))
    return lat, cost


def llama_set_method(ctx, method: int) -> None:
    _check(ctx, load().llama_set_method(ctx, int(method)))


def llama_reserve(ctx, max_inv: int) -> None:
    _check(ctx, load().llama_reserve(ctx, int(max_inv)))


def llama_schedule(ctx, dag, op_local, start_us, now_us: int, out=None):
    """Blocking call.  Host (numpy) or device (torch) arrays.  Returns (out, rc) with
    rc = OK or EINVAL (some invocations invalid, flagged in out); raises otherwise."""
    n = int(dag.shape[0])
    if out is None:
        out = np.zeros(n, dtype=DECISION_DTYPE)
    rc = load().llama_schedule(ctx, n, _ptr(dag), _ptr(op_local), _ptr(start_us), int(now_us), _ptr(out))
    _check(ctx, rc, (OK, EINVAL) if n else (OK,))
    if rc == EINVAL and "invalid" not in llama_last_error(ctx):
        raise LlamaError(rc, llama_last_error(ctx))
    return out, rc


def llama_schedule_async(ctx, dag, op_local, start_us, now_us: int, out, stream=None) -> None:
    """Enqueue on a torch CUDA stream (default: torch's current stream); device tensors only."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(ctx, load().llama_schedule_async(ctx, int(dag.shape[0]), _ptr(dag), _ptr(op_local),
                                            _ptr(start_us), int(now_us), _ptr(out),
                                            ctypes.c_void_p(stream.cuda_stream)))


STATIC_MAX_INV, STATIC_MAX_OPS = 65536, 4096


def llama_schedule_static(ctx, dag, op_local, start_us, now_us: int, out, stream=None) -> None:
    """Allocation-free scheduling call (device tensors, enqueued on a torch CUDA stream):
    the library allocates nothing during it; its scratch is one fixed device array, so
    calls must not overlap on the GPU.  At most STATIC_MAX_INV invocations and
    STATIC_MAX_OPS operations."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(ctx, load().llama_schedule_static(ctx, int(dag.shape[0]), _ptr(dag), _ptr(op_local),
                                             _ptr(start_us), int(now_us), _ptr(out),
                                             ctypes.c_void_p(stream.cuda_stream)))


def llama_static_status(ctx, stream=None) -> tuple[int, int]:
    """(invalid invocations, timeout flag) of the last completed llama_schedule_static
    call on the context's device, read on `stream` (default: torch's current stream)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    inv, tmo = ctypes.c_int64(), ctypes.c_int32()
    _check(ctx, load().llama_static_status(ctx, ctypes.c_void_p(stream.cuda_stream), ctypes.byref(inv),
                                           ctypes.byref(tmo)))
    return inv.value, tmo.value


def llama_check_word(ctx, clear: bool = True) -> int:
    """Violation bits of the checked build (LLAMA_CHECK_*; 0 in a normal build)."""
    w = ctypes.c_uint32()
    _check(ctx, load().llama_check_word(ctx, ctypes.byref(w), 1 if clear else 0))
    return w.value


def llama_set_stats_file(ctx, path) -> None:
    """Append one JSON line per blocking llama_schedule call to path (None closes it)."""
    _check(ctx, load().llama_set_stats_file(ctx, None if path is None else str(path).encode()))


def llama_set_wait_limit(ctx, tries: int) -> None:
    """Polls of a bucketing grid barrier before it gives up (WAIT_LIMIT_DEFAULT; 0 gives up at once)."""
    _check(ctx, load().llama_set_wait_limit(ctx, int(tries)))


def llama_set_direct_max(ctx, n_inv: int) -> None:
    """Scan-method calls of at most n_inv invocations skip the bucketing (DIRECT_DEFAULT; 0: never)."""
    _check(ctx, load().llama_set_direct_max(ctx, int(n_inv)))


def llama_stragglers(dec: np.ndarray, obs_us, failed, now_us: int, timeout=(3, 2), tick_us: int = 1) -> tuple:
    """(indices, hand-back times) of the invocations that get a duplicate: an
    error before the time-out or still running at it (timeout = num/den times
    the decided latency), handed back at the first tick at or after the event."""
    dec = np.ascontiguousarray(dec)
    assert dec.dtype == DECISION_DTYPE
    n = dec.shape[0]
    obs = np.ascontiguousarray(obs_us, np.int64)
    fl = None if failed is None else np.ascontiguousarray(failed, np.uint8)
    idx = np.empty(max(n, 1), np.int64)
    when = np.empty(max(n, 1), np.int64)
    k = ctypes.c_int64()
    rc = load().llama_stragglers(n, dec.ctypes.data, obs.ctypes.data, None if fl is None else fl.ctypes.data,
                                 int(now_us), int(timeout[0]), int(timeout[1]), int(tick_us), idx.ctypes.data,
                                 when.ctypes.data, ctypes.byref(k))
    if rc != OK:
        raise LlamaError(rc, "llama_stragglers failed")
    return idx[:k.value].copy(), when[:k.value].copy()


def llama_count_rate(device: int, n: int, n_counters: int) -> tuple:
    """(atomic_us, stream_us): the best time of n returning count atomics on
    n_counters counters (the bucketing kernel's counting pattern, alone) and of
    the same loads and stores without them."""
    a, b = ctypes.c_double(), ctypes.c_double()
    rc = load().llama_count_rate(int(device), int(n), int(n_counters), ctypes.byref(a), ctypes.byref(b))
    if rc != OK:
        raise LlamaError(rc, "llama_count_rate failed")
    return a.value, b.value


def llama_alu_peak(device: int = 0, mode: int = MODE_COST_FIRST) -> float:
    """Measured configurations per second of the scan's instruction mix on every SM."""
    v = ctypes.c_double()
    rc = load().llama_alu_peak(int(device), int(mode), ctypes.byref(v))
    if rc != OK:
        raise LlamaError(rc, "llama_alu_peak failed")
    return v.value


def llama_critical_path(ctx, n_ops: int) -> np.ndarray:
    cp = np.zeros(n_ops, dtype=np.int64)
    _check(ctx, load().llama_critical_path(ctx, _ptr(cp)))
    return cp


def llama_slack(ctx, dag, op_local, start_us, now_us: int, n_hw: int, out=None):
    n = int(dag.shape[0])
    if out is None:
        out = np.zeros((n, n_hw), dtype=np.int32)
    _check(ctx, load().llama_slack(ctx, n, _ptr(dag), _ptr(op_local), _ptr(start_us), int(now_us),
                                   _ptr(out)))
    return out


def llama_set_trace_events(ctx, events) -> None:
    """events: list of TRACE_EVENTS torch.cuda.Event(enable_timing=True), or [] to stop."""
    if not events:
        _check(ctx, load().llama_set_trace_events(ctx, None, 0))
        return
    for e in events:
        if not e.cuda_event:  # torch creates the handle on first record
            e.record()
    arr = (ctypes.c_void_p * len(events))(*[e.cuda_event for e in events])
    _check(ctx, load().llama_set_trace_events(ctx, arr, len(events)))


def llama_last_launch_count(ctx) -> int:
    return load().llama_last_launch_count(ctx)


class Loop:
    """The device-resident serving loop (early speculation and late commit,
    priority-based commit) over a Scheduler's context."""

    def __init__(self, sched, slots: int = 65536, ring: int = 1 << 16, results: int = 1 << 18,
                 max_admit: int = 1024, cq_cap=(64, 64, 64)):
        self.lib = load()
        self.sched = sched
        opts = llama_loop_opts(slots, ring, results, max_admit, (ctypes.c_int32 * MAX_HW)(*cq_cap))
        h = ctypes.c_void_p()
        _check(sched.ctx, self.lib.llama_loop_create(sched.ctx, ctypes.byref(opts), ctypes.byref(h)))
        self.h = h
        self.n_hw = sched.problem.n_hw
        self._buf = np.zeros(max(results, 1), LOOP_RESULT_DTYPE)

    def _check(self, rc):
        _check(self.sched.ctx, rc)

    def submit(self, req: np.ndarray) -> int:
        req = np.ascontiguousarray(req, LOOP_REQUEST_DTYPE)
        rc = self.lib.llama_loop_submit(self.h, req.ctypes.data, req.shape[0])
        if rc not in (OK, EAGAIN):
            self._check(rc)
        return rc

    def tick(self, now_us: int, dispatch=None) -> None:
        d = None if dispatch is None else np.ascontiguousarray(dispatch, np.int32)
        self._check(self.lib.llama_loop_tick(self.h, int(now_us), None if d is None else d.ctypes.data))

    def poll(self) -> np.ndarray:
        n = ctypes.c_int64()
        self._check(self.lib.llama_loop_poll(self.h, self._buf.ctypes.data, self._buf.shape[0], ctypes.byref(n)))
        return self._buf[:n.value].copy()

    def sync(self) -> None:
        self._check(self.lib.llama_loop_sync(self.h))

    def ticks_done(self) -> int:
        return int(self.lib.llama_loop_ticks_done(self.h))

    def start(self, now_us: int, ticks_in_flight: int = 2, dispatch=None) -> None:
        """Ticks on the library's driver thread (dispatch: per-tick counts; None =
        dispatch every commit queue whole each tick)."""
        d = np.full(self.n_hw, 2**31 - 1, np.int32) if dispatch is None else np.ascontiguousarray(dispatch, np.int32)
        self._dispatch = d
        self._check(self.lib.llama_loop_start(self.h, int(now_us), int(ticks_in_flight), d.ctypes.data))

    def stop(self) -> None:
        self._check(self.lib.llama_loop_stop(self.h))

    def run_arrivals(self, req: np.ndarray, arrive_ns: np.ndarray, timeout_s: float = 10.0) -> tuple:
        """Submit req[k] at arrive_ns[k] (ns after the call starts) and poll, on a
        native host thread (the driver must run): (spec_ns, commit_ns), when each
        request's records were seen (-1 if not)."""
        req = np.ascontiguousarray(req, LOOP_REQUEST_DTYPE)
        t = np.ascontiguousarray(arrive_ns, np.int64)
        n = req.shape[0]
        spec = np.empty(max(n, 1), np.int64)
        com = np.empty(max(n, 1), np.int64)
        id0 = int(req["id"][0]) if n else 0
        self._check(self.lib.llama_loop_run_arrivals(self.h, req.ctypes.data, t.ctypes.data, n, id0,
                                                     int(timeout_s * 1e9), spec.ctypes.data, com.ctypes.data))
        return spec[:n], com[:n]

    def state(self) -> dict:
        st = llama_loop_state()
        self._check(self.lib.llama_loop_state_get(self.h, ctypes.byref(st)))
        H = self.n_hw
        return {"ticks": st.ticks, "submitted": st.submitted, "admitted": st.admitted, "rejected": st.rejected,
                "committed": st.committed, "dispatched": st.dispatched, "results": st.results,
                "results_dropped": st.results_dropped, "free_slots": st.free_slots,
                "sq_len": list(st.sq_len)[:H], "cq_len": list(st.cq_len)[:H], "q_us": list(st.q_us)[:H]}

    def refresh(self) -> None:
        self._check(self.lib.llama_loop_refresh(self.h))

    def close(self) -> None:
        if self.h:
            self.lib.llama_loop_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Scheduler:
    """A context loaded with one Problem (see ``workloads``).  direct_max: the
    small-call limit (llama_set_direct_max; None keeps the class attribute,
    whose None keeps the library's DIRECT_DEFAULT)."""

    direct_max = None

    def __init__(self, problem, mode: int = MODE_COST_FIRST, alpha=(1, 1), device: int = 0,
                 use_graph: bool = False, method: int = METHOD_SCAN, direct_max=None):
        self.problem = problem
        self.mode = mode
        self.ctx = llama_create(mode, problem.n_hw, alpha, device, use_graph)
        if method != METHOD_SCAN:
            llama_set_method(self.ctx, method)
        direct_max = self.direct_max if direct_max is None else direct_max
        if direct_max is not None:
            llama_set_direct_max(self.ctx, direct_max)
        p = problem
        llama_set_dags(self.ctx, p.dag_op_off, p.row_ptr, p.col, p.slo_us)
        alpha_mode = mode == MODE_ALPHA
        with_res = alpha_mode or (p.batch is not None and p.res is not None and p.res_total is not None)
        llama_set_profiles(self.ctx, p.cfg_off, p.hw_off, p.lat_us, p.cost_nd, p.ref_cfg,
                           p.batch if with_res else None, p.res if with_res else None,
                           p.res_total if with_res else None)
        if p.q_us is not None:
            llama_set_queue(self.ctx, p.q_us)

    def schedule(self, inv, out=None):
        return llama_schedule(self.ctx, _c(inv.dag, np.int32), _c(inv.op_local, np.int32),
                              _c(inv.start_us, np.int64), inv.now_us, out)

    def slack(self, inv):
        return llama_slack(self.ctx, _c(inv.dag, np.int32), _c(inv.op_local, np.int32),
                           _c(inv.start_us, np.int64), inv.now_us, self.problem.n_hw)

    def critical_path(self):
        return llama_critical_path(self.ctx, self.problem.n_ops)

    def close(self):
        if self.ctx:
            llama_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
