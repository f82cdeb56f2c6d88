"""The learned latency surrogate: features, training and scheduling, on the GPU.

Argument marshalling around the C ABI of ``include/llama_surrogate.h``: the
network's forward and backward passes, the optimizer and the scheduling with
predicted latencies all run in the library's kernels.  Training data are the
profiler's samples (``workloads.surrogate_training_set``).
"""
from __future__ import annotations

import contextlib
import ctypes

import numpy as np

from . import llama as L
from . import workloads as W


def _bf16(x: np.ndarray, col0: int, device="cuda"):
    import torch
    out = np.zeros((x.shape[0], L.MLP_INPUTS), np.float32)
    out[:, col0:col0 + x.shape[1]] = x
    return torch.from_numpy(out).to(device).to(torch.bfloat16)


def config_inputs(p, cw, device="cuda"):
    """Features of every configuration of p (row = global configuration), BF16 [n_cfg, 64]."""
    sizes = np.diff(p.cfg_off)
    gop = np.repeat(np.arange(p.n_ops), sizes)
    cfg = np.arange(p.n_cfg) - np.repeat(p.cfg_off[:-1], sizes)
    return _bf16(W.config_features(p, cw, gop, cfg), 0, device)


def content_inputs(content, device="cuda"):
    """Features of invocation content, BF16 [n, 64] in columns 32..47."""
    return _bf16(W.content_features(content), W.N_CFG_FEATURES, device)


def training_inputs(x: np.ndarray, t: np.ndarray, device="cuda"):
    import torch
    return _bf16(x, 0, device), torch.from_numpy(np.ascontiguousarray(t, np.float32)).to(device)


def _run_epochs(net, x, t, batch: int, w_fan: float, plan, stream=None) -> list:
    """Adam epochs over the device tensors x (BF16 [n, 64]) and t (FP32 [n, 2]):
    plan yields (permutation of the rows, CPU tensor; learning rate) per epoch,
    lazily, so that the next epoch's order is drawn on the host and copied while
    the current epoch runs.  The epochs' mean batch losses."""
    import torch
    nb = x.shape[0] // batch
    acc = torch.zeros(1, dtype=torch.float32, device=x.device)
    history = []

    def upload(item):
        if item is None:
            return None
        perm, lr = item
        host = perm[:nb * batch].to(torch.int32).pin_memory()
        return host, host.to(x.device, non_blocking=True), lr

    plan = iter(plan)
    # the permutation, the loss sum and the epochs on one stream
    with torch.cuda.stream(stream) if stream is not None else contextlib.nullcontext():
        nxt = upload(next(plan, None))
        while nxt is not None:
            _, perm, lr = nxt
            acc.zero_()
            # every batch of the epoch in one library call: gathered on the device
            net.train_epoch(x, t, perm, batch, w_fan, lr, acc, stream)
            nxt = upload(next(plan, None))  # drawn and copied while this epoch runs
            history.append(float(acc.item()) / nb)
    return history


def train(net, x, t, epochs: int, batch: int = 8192, lr: float = 1e-3, w_fan: float = 0.5, seed: int = 0,
          stream=None) -> list:
    """Adam over shuffled mini-batches of the device tensors x (BF16 [n, 64]) and
    t (FP32 [n, 2]), one seeded generator for every epoch's order; the mean
    batch loss of every epoch."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    plan = ((torch.randperm(x.shape[0], generator=g), lr) for _ in range(epochs))
    return _run_epochs(net, x, t, batch, w_fan, plan, stream)


def held_out_rmse(net, x, t, batch: int = 8192) -> float:
    """Root mean square error of the first output on held-out device tensors."""
    import torch
    y = torch.empty(x.shape[0], 2, dtype=torch.float32, device=x.device)
    for i in range(0, x.shape[0], batch):
        net.forward(x[i:i + batch].contiguous(), y[i:i + batch])
    return float(torch.sqrt(torch.mean((y[:, 0] - t[:, 0]) ** 2)).item())


def margin_from_rmse(rmse: float, noise_sigma: float) -> float:
    """The model's own error from the held-out error and the profiler's known
    measurement noise (independent errors add in variance), used as the
    selection margin (at most 1, the largest margin the scheduler takes)."""
    return float(min(np.sqrt(max(rmse * rmse - noise_sigma * noise_sigma, 0.0)), 1.0))


def train_schedule(net, x, t, epochs: int = 12, lr: float = 2e-3, halve_every: int = 3, w_fan: float = 0.1,
                   seed: int = 0) -> list:
    """Adam with the learning rate halved every few epochs (epoch e's order from a
    generator seeded seed + e); the epochs' mean losses."""
    import torch

    def order(e):
        return torch.randperm(x.shape[0], generator=torch.Generator(device="cpu").manual_seed(seed + e))

    plan = ((order(e), lr * 0.5 ** (e // halve_every)) for e in range(epochs))
    return _run_epochs(net, x, t, 8192, w_fan, plan)


class SurrogateScheduler:
    """Scheduling with the network's predictions on a context's problem."""

    def __init__(self, sched, net, max_inv: int, max_pairs: int):
        self.sched, self.net = sched, net
        self.h = ctypes.c_void_p()
        rc = L.load().llama_sg_create(ctypes.byref(self.h), sched.ctx, net.h, int(max_inv), int(max_pairs))
        if rc != L.OK:
            raise L.LlamaError(rc, "sg_create failed")

    def _check(self, rc):
        if rc != L.OK:
            raise L.LlamaError(rc, L.load().llama_sg_last_error(self.h).decode())

    def set_margin(self, margin: float) -> None:
        self._check(L.load().llama_sg_set_margin(self.h, float(margin)))

    def invalidate(self) -> None:
        """Recompute layer 1's configuration part at the next call (after the
        configuration features changed in place)."""
        self._check(L.load().llama_sg_invalidate(self.h))

    def schedule_device(self, cfg_x, inv_x, dag, op_local, start, now_us: int, out, stream=None) -> None:
        v = lambda t: ctypes.c_void_p(t.data_ptr())
        self._check(L.load().llama_sg_schedule(self.h, v(cfg_x), v(inv_x), dag.shape[0], v(dag), v(op_local),
                                               v(start), int(now_us), v(out), L._stream_ptr(stream)))

    def run_arrivals(self, cfg_x, inv_x, dag, op_local, start, arrive_ns, now_us: int, max_batch: int = 4096,
                     stream=None):
        """Continuous batching on a native host thread: each call takes every
        request that arrived while the previous one ran (at most max_batch);
        returns when each request's decision was back on the host (ns after the
        start).  inv_x, dag, op_local, start: device tensors, one row per request."""
        import torch
        v = lambda t: ctypes.c_void_p(t.data_ptr())
        n = dag.shape[0]
        t = np.ascontiguousarray(arrive_ns, np.int64)
        out = torch.zeros(max_batch * 24, dtype=torch.uint8, device=dag.device)
        host = torch.zeros(max_batch * 24, dtype=torch.uint8).pin_memory()
        done = np.full(max(n, 1), -1, np.int64)
        self._check(L.load().llama_sg_run_arrivals(self.h, v(cfg_x), v(inv_x), v(dag), v(op_local), v(start), n,
                                                   t.ctypes.data, int(now_us), int(max_batch), v(out), v(host),
                                                   L._stream_ptr(stream), done.ctypes.data))
        return done[:n]

    def schedule(self, cfg_x, inv, content):
        """Decisions (numpy, DECISION_DTYPE) for invocations with their content."""
        import torch
        dev = cfg_x.device
        dag = torch.from_numpy(inv.dag).to(dev)
        opl = torch.from_numpy(inv.op_local).to(dev)
        st = torch.from_numpy(inv.start_us).to(dev)
        out = torch.zeros(inv.n * 24, dtype=torch.uint8, device=dev)
        self.schedule_device(cfg_x, content_inputs(content, dev), dag, opl, st, inv.now_us, out)
        torch.cuda.synchronize()
        return out.cpu().numpy().view(L.DECISION_DTYPE)

    def predictions(self, n_inv: int):
        """Predicted latency and cost of every pair of the last call, and the pair offsets."""
        import torch
        n = int(L.load().llama_sg_last_pairs(self.h))
        lh = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
        ch = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
        po = torch.empty(n_inv + 1, dtype=torch.int64, device="cuda")
        v = lambda t: ctypes.c_void_p(t.data_ptr())
        self._check(L.load().llama_sg_predictions(self.h, v(lh), v(ch), v(po), n_inv, L._stream_ptr(None)))
        torch.cuda.synchronize()
        return lh[:n].cpu().numpy(), ch[:n].cpu().numpy(), po.cpu().numpy()

    def close(self):
        if self.h:
            L.load().llama_sg_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
