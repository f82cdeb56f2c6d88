"""The surrogate network's CUDA kernels (forward, gradients, Adam) against
the FP64 oracle of the same network (oracle/mlp.py)."""
import numpy as np
import pytest

from oracle import mlp as M
from paper_2102_01887_b300 import workloads as W
from tests import bf16_bounds as BB

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L(cuda_device):
    from paper_2102_01887_b300 import build, llama
    build.build()
    llama.load()
    return llama


def bf16_round(a):
    import torch
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


@pytest.fixture(scope="module")
def world():
    p, _ = W.medium()
    cw = W.content_world(p)
    x, t = W.surrogate_training_set(p, cw, 400_000, seed=7)
    return p, cw, x, t


def perturbed_params(seed):
    rng = np.random.default_rng(seed)
    p = M.init_params(seed)
    for k in p:
        if k in ("W4", "b4"):
            p[k][:2] += rng.normal(0, 0.05, p[k][:2].shape)
        else:
            p[k] += rng.normal(0, 0.02, p[k].shape)
    return p


def to_device_x(x):
    import torch
    xp = np.zeros((x.shape[0], M.IN), np.float32)
    xp[:, :x.shape[1]] = x
    return torch.from_numpy(xp).to(torch.bfloat16).cuda()


def rounded(p):
    """The parameters as the GPU multiplies them: weights in BF16, biases in FP32."""
    return {k: bf16_round(v) if k.startswith("W") else v for k, v in p.items()}


def test_forward_matches_oracle(L, world):
    import torch
    _, _, x, _ = world
    p = perturbed_params(1)
    xs = x[:3000]
    with L.MLP(max_batch=4096) as net:
        net.set_params(M.pack(p).astype(np.float32))
        xd = to_device_x(xs)
        y = torch.empty(xs.shape[0], 2, dtype=torch.float32, device="cuda")
        net.forward(xd, y)
        got = y.cpu().numpy()
    q = rounded(M.unpack(M.pack(p).astype(np.float32)))
    y, sy, _, _ = BB.forward_errors(q, bf16_round(M.pad_features(xs)))
    ref, tol = y[:, :2], BB.tol(sy)[:, :2]
    # element by element, within the tolerance derived from BF16 rounding
    # (tests/bf16_bounds.py: 8 sigma of the propagated rounding error)
    bad = np.abs(got - ref) > tol
    assert not bad.any(), (int(bad.sum()), float((np.abs(got - ref) / tol).max()))
    scale = np.abs(ref).max(axis=0) + 1e-3
    assert (np.abs(got - ref) / scale).max() < 0.03, (np.abs(got - ref) / scale).max()


def test_gradients_match_oracle(L, world):
    import torch
    _, _, x, t = world
    p = perturbed_params(2)
    n = 512
    xs, ts = x[:n], t[:n]
    w_fan = 0.5
    with L.MLP(max_batch=1024) as net:
        net.set_params(M.pack(p).astype(np.float32))
        g = torch.empty(M.N_PARAMS, dtype=torch.float32, device="cuda")
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        net.gradients(to_device_x(xs), torch.from_numpy(ts).cuda(), w_fan, g, loss)
        got = M.unpack(g.cpu().numpy().astype(np.float64))
        got_loss = float(loss.item())
    q = rounded(M.unpack(M.pack(p).astype(np.float32)))
    ref_loss, ref, tol = BB.gradient_errors(q, bf16_round(M.pad_features(xs)), ts.astype(np.float64), w_fan)
    assert got_loss == pytest.approx(ref_loss, rel=0.02)
    for name, _ in M.SHAPES:
        a, b, e = got[name], ref[name], tol[name]
        if name in ("W4", "b4"):
            a, b, e = a[:2], b[:2], e[:2]
            assert not got[name][2:].any()  # outputs the loss never reads
        # element by element, within the tolerance derived from BF16 rounding
        bad = np.abs(a - b) > e + 1e-30
        assert not bad.any(), (name, int(bad.sum()), float((np.abs(a - b) / (e + 1e-30)).max()))
        rel = np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-12)
        assert rel < 0.05, (name, rel)


def test_adam_step_matches_oracle_update(L, world):
    import torch
    _, _, x, t = world
    p = perturbed_params(3)
    n = 256
    xs, ts = to_device_x(x[:n]), torch.from_numpy(t[:n]).cuda()
    lr = 1e-3
    with L.MLP(max_batch=256) as net:
        flat = M.pack(p).astype(np.float32)
        net.set_params(flat)
        g = torch.empty(M.N_PARAMS, dtype=torch.float32, device="cuda")
        net.gradients(xs, ts, 1.0, g)
        net.train_step(xs, ts, 1.0, lr)
        after = net.get_params().astype(np.float64)
    q = M.unpack(flat.astype(np.float64))
    gg = M.unpack(g.cpu().numpy().astype(np.float64))
    m = {k: np.zeros_like(v) for k, v in q.items()}
    v = {k: np.zeros_like(v) for k, v in q.items()}
    M.adam_step(q, gg, m, v, 1, lr)
    exp = M.pack(q)
    # first step: lr * g / (|g| + eps); gradients may differ in the last bits (atomic order)
    assert np.abs(after - exp).max() <= 2e-3 * lr + 1e-6


def test_training_reduces_the_loss(L, world):
    import torch
    _, _, x, t = world
    n_train = 380_000
    xt, tt = to_device_x(x[:n_train]), torch.from_numpy(t[:n_train]).cuda()
    xv, tv = x[n_train:], t[n_train:]
    batch = 8192
    with L.MLP(max_batch=batch) as net:
        net.set_params(M.pack(M.init_params(11)).astype(np.float32))
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        first = None
        rng = np.random.default_rng(0)
        for epoch in range(4):
            perm = torch.from_numpy(rng.permutation(n_train)).cuda()
            for b in range(n_train // batch):
                idx = perm[b * batch:(b + 1) * batch]
                net.train_step(xt[idx].contiguous(), tt[idx].contiguous(), 0.5, 1e-3, loss)
                if first is None:
                    first = float(loss.item())
        torch.cuda.synchronize()
        assert L.llama_gemm_error(True) == L.OK
        xvd = to_device_x(xv)
        y = torch.empty(xv.shape[0], 2, dtype=torch.float32, device="cuda")
        for i in range(0, xv.shape[0], batch):
            net.forward(xvd[i:i + batch].contiguous(), y[i:i + batch])
        pred = y.cpu().numpy()
    # the latency factor: most of its variance explained (noise sigma 0.1 of 0.55)
    r2 = 1 - np.mean((pred[:, 0] - tv[:, 0]) ** 2) / np.var(tv[:, 0])
    assert r2 > 0.85, r2
    assert float(loss.item()) < 0.3 * first


def test_train_epoch_equals_the_same_steps_one_at_a_time(L, world):
    """llama_mlp_train_epoch (batches gathered on the device, no host round
    trip per step) leaves the parameters equal to those of the same batches
    taken one llama_mlp_train_step at a time, and sums the same batch losses;
    an out-of-range index gives a zero row.  Equal up to the order of the
    bias gradients' atomic sums: nearly every parameter to the last bits, and
    none further apart than the steps' learning rate can move it."""
    import torch
    _, _, x, t = world
    n_rows, batch, n_batches = 40_000, 1024, 6
    xd, td = to_device_x(x[:n_rows]), torch.from_numpy(t[:n_rows]).cuda()
    perm = torch.from_numpy(np.random.default_rng(5).permutation(n_rows)[:batch * n_batches].astype(np.int32)).cuda()
    start = M.pack(perturbed_params(9)).astype(np.float32)
    with L.MLP(max_batch=batch) as a, L.MLP(max_batch=batch) as b:
        a.set_params(start)
        b.set_params(start)
        la = torch.zeros(1, dtype=torch.float32, device="cuda")
        a.train_epoch(xd, td, perm, batch, 0.5, 1e-3, la)
        lb, one = torch.zeros(1, dtype=torch.float32, device="cuda"), torch.zeros(1, dtype=torch.float32, device="cuda")
        for k in range(n_batches):
            idx = perm[k * batch:(k + 1) * batch].long()
            b.train_step(xd[idx].contiguous(), td[idx].contiguous(), 0.5, 1e-3, one)
            lb += one
        def assert_close(pa, pb, steps):
            d = np.abs(pa.astype(np.float64) - pb)
            assert np.mean(d <= 1e-6 * np.abs(pb) + 1e-9) > 0.999, float(d.max())
            assert d.max() <= 2 * 1e-3 * steps
        assert_close(a.get_params(), b.get_params(), n_batches)
        assert abs(float(la.item()) - float(lb.item())) <= 1e-5 * abs(float(lb.item()))
        # a zero row for an index outside the rows: same as a batch with that row zeroed
        bad = perm[:batch].clone()
        bad[7] = n_rows + 3
        a.set_params(start)
        b.set_params(start)
        a.train_epoch(xd, td, bad, batch, 0.5, 1e-3)
        idx = bad.long().clamp(max=n_rows - 1)
        xz, tz = xd[idx].contiguous(), td[idx].contiguous()
        xz[7].zero_()
        tz[7].zero_()
        b.train_step(xz, tz, 0.5, 1e-3)
        assert_close(a.get_params(), b.get_params(), 1)
        with pytest.raises(L.LlamaError):
            a.train_epoch(xd, td, perm[:2000], 1000, 0.5, 1e-3)  # not a multiple of 128
