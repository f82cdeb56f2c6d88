"""Scheduling with the learned latency surrogate.

Parity: the predicted latencies of every (invocation, configuration) pair
against the FP64 oracle of the network (a tolerance from BF16 activations:
|log(predicted / oracle)| <= 0.05), and every decision bit-exact against the
oracle's selection rule applied to the GPU's own integer predictions.
Evaluation: after training on the profiler's samples, decisions judged on the
ground-truth content model against the profile-table path.
"""
import numpy as np
import pytest

import oracle
from oracle import mlp as M
from tests import bf16_bounds as BB
from oracle import surrogate as OS
from paper_2102_01887_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L(cuda_device):
    from paper_2102_01887_b300 import build, llama
    build.build()
    llama.load()
    return llama


@pytest.fixture(scope="module")
def world():
    p, inv = W.medium()
    return p, inv, W.content_world(p)


def pairs_of(p, inv, valid):
    """Pair layout: invocation, global configuration, op-local index, offsets."""
    gop = p.dag_op_off[np.where(valid, inv.dag, 0)] + np.where(valid, inv.op_local, 0)
    sizes = np.where(valid, np.diff(p.cfg_off)[gop], 0)
    off = np.zeros(inv.n + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    pinv = np.repeat(np.arange(inv.n), sizes)
    px = np.arange(off[-1]) - np.repeat(off[:-1], sizes)
    pg = p.cfg_off[gop[pinv]] + px
    return pinv, pg, px, off, gop


def backend_of_cfg(p):
    lam = np.zeros(p.n_cfg, np.int64)
    hw = p.hw_off.reshape(p.n_ops, p.n_hw + 1)
    for v in range(p.n_ops):
        for h in range(p.n_hw):
            lam[p.cfg_off[v] + hw[v, h]:p.cfg_off[v] + hw[v, h + 1]] = h
    return lam


def perturbed_params(seed):
    rng = np.random.default_rng(seed)
    q = M.init_params(seed)
    for k in q:
        q[k] = q[k] + (rng.normal(0, 0.05, q[k].shape) if k in ("W4", "b4") else rng.normal(0, 0.02, q[k].shape))
    q["W4"][2:] = 0
    q["b4"][2:] = 0
    return q


def check_predictions(L, p, sub, cw, seed):
    """Predictions and decisions of the GPU against the oracle on the invocations
    sub (two of them made invalid) with random content and perturbed weights."""
    import torch

    from paper_2102_01887_b300 import surrogate as S
    sub.dag = sub.dag.copy()
    sub.start_us = sub.start_us.copy()
    sub.dag[3] = -1
    sub.start_us[7] = sub.now_us + 5
    content = W.invocation_content(seed, sub.n)
    params = perturbed_params(seed + 16)
    flat = M.pack(params).astype(np.float32)
    slack = oracle.slacks(p, sub)
    valid = slack[:, 0] >= 0
    pinv, pg, px, off, gop = pairs_of(p, sub, valid)
    with L.Scheduler(p) as s, L.MLP(max_batch=1024) as net:
        net.set_params(flat)
        cfg_x = S.config_inputs(p, cw)
        with S.SurrogateScheduler(s, net, max_inv=4096, max_pairs=1 << 20) as sg:
            got = sg.schedule(cfg_x, sub, content)
            lh, ch, po = sg.predictions(sub.n)
        # the features of the configurations that occur, rows renumbered
        used, pg_used = np.unique(pg, return_inverse=True)
        cfg_np = cfg_x[torch.from_numpy(used).to(cfg_x.device)].float().cpu().numpy()
        inv_np = S.content_inputs(content).float().cpu().numpy()
    assert (got["flags"][~valid] == L.FLAG_INVALID).all() and (got["cfg"][~valid] == -1).all()
    assert np.array_equal(po, off)
    # the network, in FP64 on the same BF16 inputs and weights (last layer in FP32)
    q = M.unpack(flat.astype(np.float64))
    for k in ("W1", "W2", "W3"):
        q[k] = torch.from_numpy(q[k].astype(np.float32)).to(torch.bfloat16).double().numpy()
    r = OS.forward_log_factor(q, cfg_np, inv_np, pinv, pg_used)
    l_or = p.lat_us[pg] * np.exp(np.clip(r, -20, 20))
    err = np.abs(np.log(lh / l_or))
    assert err.max() <= 0.05, err.max()
    # element by element: the log factor within the tolerance derived from BF16
    # rounding of the split first layer, h1 and h2 (tests/bf16_bounds.py), plus
    # expf (a few float ulps) and the rounding of L e^r to whole microseconds
    x_cfg = np.zeros((pinv.shape[0], M.IN))
    x_cfg[:, :32] = cfg_np[pg_used, :32]
    x_inv = np.zeros((pinv.shape[0], M.IN))
    x_inv[:, 32:48] = inv_np[pinv, 32:48]
    y0, tol = BB.split_forward_errors(q, x_cfg, x_inv)
    assert np.allclose(y0, r)
    bound = tol + 1e-6 + 0.5 / np.maximum(lh - 0.5, 0.5)
    bad = err > bound
    assert not bad.any(), (int(bad.sum()), float((err / bound).max()))
    # selection: the oracle's rule on the GPU's integer predictions
    lam = backend_of_cfg(p)
    spair = slack[pinv, lam[pg]]
    x_or = OS.select(lh.astype(np.int64), ch, spair, off)
    assert np.array_equal(got["cfg"][valid], x_or[valid])
    k = off[:-1][valid] + x_or[valid]
    assert np.array_equal(got["lat"][valid], lh[k])
    assert np.array_equal(got["cost"][valid], ch[k])
    assert np.array_equal(got["slack"][valid], spair[k])
    assert np.array_equal(got["flags"][valid], (lh[k] < spair[k]).astype(np.int32))


def test_predictions_and_decisions_match_oracle(L, world):
    p, inv, cw = world
    check_predictions(L, p, inv.subset(np.arange(0, inv.n, 640)), cw, 5)


def test_predictions_uneven_configuration_spaces(L):
    """Zipf-sized configuration spaces (96 .. 8,192, most not a multiple of the
    128-row tile): every invocation's last tile is partly padding."""
    p, inv = W.batched(n_inv=4096)
    sizes = np.diff(p.cfg_off)[p.dag_op_off[inv.dag] + inv.op_local]
    assert (sizes % 128 != 0).mean() > 0.3
    check_predictions(L, p, inv.subset(np.arange(0, inv.n, 29)), W.content_world(p), 7)


def evaluate(p, cw, sub, content, decisions_cfg, slack, lam, noise_seed):
    """True latency / cost of each invocation's chosen configuration, with the
    ground-truth content model and its lognormal noise."""
    valid = slack[:, 0] >= 0
    pinv, pg, px, off, gop = pairs_of(p, sub, valid)
    ci = W.Content(content.n_obj[pinv], content.motion[pinv], content.in_res[pinv])
    f = W.true_log_factor(p, cw, gop[pinv], px, ci) + W.latency_noise(noise_seed, pinv.shape[0])
    lt = np.maximum(1, np.rint(p.lat_us[pg] * np.exp(f))).astype(np.int64)
    ct = np.rint(p.cost_nd[pg] * np.exp(f)).astype(np.int64)
    spair = slack[pinv, lam[pg]]
    best = OS.select(lt, ct, spair, off)
    res = {}
    for name, x in list(decisions_cfg.items()) + [("truth", best)]:
        k = off[:-1][valid] + x[valid]
        viol = lt[k] >= spair[k]
        res[name] = {"violations": float(viol.mean()), "cost": float(ct[k].sum()), "cfg": x[valid]}
    return res


def test_layer1_configuration_part_is_kept_while_valid(L, world):
    """Layer 1's configuration part is computed once and kept across calls; a
    weight change (set_params) or llama_sg_invalidate after an in-place change
    of the features makes the next call recompute it.  Every call must equal a
    fresh scheduler's."""
    import torch

    from paper_2102_01887_b300 import surrogate as S
    p, inv, cw = world
    sub = inv.subset(np.arange(0, inv.n, 512))
    content = W.invocation_content(3, sub.n)
    with L.Scheduler(p) as s, L.MLP(max_batch=1024) as net:
        cfg_x = S.config_inputs(p, cw)

        def fresh():
            with S.SurrogateScheduler(s, net, max_inv=4096, max_pairs=1 << 20) as f:
                return f.schedule(cfg_x, sub, content)

        with S.SurrogateScheduler(s, net, max_inv=4096, max_pairs=1 << 20) as sg:
            net.set_params(M.pack(perturbed_params(21)).astype(np.float32))
            a = sg.schedule(cfg_x, sub, content)
            assert np.array_equal(sg.schedule(cfg_x, sub, content), a)  # kept
            assert np.array_equal(a, fresh())
            net.set_params(M.pack(perturbed_params(22)).astype(np.float32))  # new weights
            b = sg.schedule(cfg_x, sub, content)
            assert np.array_equal(b, fresh()) and not np.array_equal(b, a)
            # features changed in place: stale until invalidated
            cfg_x[:, :32] = torch.flip(cfg_x[:, :32], dims=[0])
            sg.invalidate()
            assert np.array_equal(sg.schedule(cfg_x, sub, content), fresh())


def test_decisions_are_the_same_alone_and_in_any_mix(L, world):
    """Serving batches whatever has arrived: an invocation's surrogate decision
    must not depend on the batch it lands in.  Every pair row is computed on its
    own (its own inputs, the same weights and summation order) and the
    per-invocation minimum is order-free, so decisions are bit-identical alone,
    in one batch, and in a shuffled batch with other invocations."""
    from paper_2102_01887_b300 import surrogate as S
    p, inv, cw = world
    sub = inv.subset(np.arange(0, inv.n, 1024))  # 64 invocations
    content = W.invocation_content(4, sub.n)
    with L.Scheduler(p) as s, L.MLP(max_batch=1024) as net:
        net.set_params(M.pack(perturbed_params(31)).astype(np.float32))
        cfg_x = S.config_inputs(p, cw)
        with S.SurrogateScheduler(s, net, max_inv=4096, max_pairs=1 << 20) as sg:
            sg.set_margin(0.02)
            together = sg.schedule(cfg_x, sub, content)
            alone = np.concatenate([sg.schedule(cfg_x, sub.subset(np.asarray([i])),
                                                W.Content(content.n_obj[i:i + 1], content.motion[i:i + 1],
                                                          content.in_res[i:i + 1]))
                                    for i in range(sub.n)])
            rng = np.random.default_rng(2)
            other = inv.subset(rng.integers(0, inv.n, 500))
            oc = W.invocation_content(5, other.n)
            mix_idx = rng.permutation(sub.n + other.n)
            dag = np.concatenate([sub.dag, other.dag])[mix_idx]
            opl = np.concatenate([sub.op_local, other.op_local])[mix_idx]
            st = np.concatenate([sub.start_us, other.start_us])[mix_idx]
            mc = W.Content(*(np.concatenate([getattr(content, k), getattr(oc, k)])[mix_idx]
                             for k in ("n_obj", "motion", "in_res")))
            mixed = sg.schedule(cfg_x, W.Invocations(dag, opl, st, sub.now_us), mc)
            back = np.empty(sub.n, dtype=mixed.dtype)
            pos = np.argsort(mix_idx)[:sub.n]  # where each of sub's invocations went
            back[:] = mixed[pos]
    for k in ("cfg", "lat", "cost", "slack", "flags"):
        assert np.array_equal(together[k], alone[k]), k
        assert np.array_equal(together[k], back[k]), k


@pytest.mark.slow
def test_edge_cases(L, world):
    """A single invocation; a call in which every invocation is invalid (no pair
    rows: only the decode runs); more pairs than max_pairs; predictions asked
    for another invocation count than the last call's."""
    from paper_2102_01887_b300 import surrogate as S
    p, inv, cw = world
    params = perturbed_params(33)
    flat = M.pack(params).astype(np.float32)
    with L.Scheduler(p) as s, L.MLP(max_batch=1024) as net:
        net.set_params(flat)
        cfg_x = S.config_inputs(p, cw)
        with S.SurrogateScheduler(s, net, max_inv=64, max_pairs=4096) as sg:
            one = inv.subset(np.array([5]))
            got = sg.schedule(cfg_x, one, W.invocation_content(3, 1))
            lh, ch, po = sg.predictions(1)
            n = int(np.diff(p.cfg_off)[p.dag_op_off[one.dag[0]] + one.op_local[0]])
            assert po.tolist() == [0, n] and lh.shape == (n,)
            x = OS.select(lh.astype(np.int64), ch,
                          oracle.slacks(p, one)[0][backend_of_cfg(p)[p.cfg_off[p.dag_op_off[one.dag[0]] +
                                                                           one.op_local[0]] + np.arange(n)]],
                          po)
            assert got["cfg"][0] == x[0]
            with pytest.raises(L.LlamaError):
                sg.predictions(2)
            bad = inv.subset(np.arange(8))
            bad.dag = np.full(8, -1, np.int32)
            got = sg.schedule(cfg_x, bad, W.invocation_content(4, 8))
            assert (got["flags"] == L.FLAG_INVALID).all() and (got["cfg"] == -1).all()
            lh, ch, po = sg.predictions(8)
            assert lh.shape == (0,) and (po == 0).all()
            many = inv.subset(np.arange(16))  # 16 x 1,024 pairs > 4,096
            with pytest.raises(L.LlamaError):
                sg.schedule(cfg_x, many, W.invocation_content(5, 16))


def test_trained_surrogate_against_the_table_path(L, world):
    # trained on 2M profiler samples, margin from the held-out error, judged on
    # 16,384 invocations with the ground-truth content model
    from paper_2102_01887_b300 import surrogate as S
    p, inv, cw = world
    x, t = W.surrogate_training_set(p, cw, 2_000_000)
    xv, tv = W.surrogate_training_set(p, cw, 100_000, seed=303)
    sub = inv.subset(np.arange(0, inv.n, 4))
    slack = oracle.slacks(p, sub)
    lam = backend_of_cfg(p)
    with L.Scheduler(p) as s, L.MLP(max_batch=8192) as net:
        net.set_params(M.pack(M.init_params(3)).astype(np.float32))
        xd, td = S.training_inputs(x, t)
        hist = S.train_schedule(net, xd, td)
        rmse = S.held_out_rmse(net, *S.training_inputs(xv, tv))
        margin = S.margin_from_rmse(rmse, W.LATENCY_NOISE_SIGMA)
        cfg_x = S.config_inputs(p, cw)
        out = {}
        with S.SurrogateScheduler(s, net, max_inv=sub.n, max_pairs=sub.n * 1024) as sg:
            sg.set_margin(margin)
            table, _ = s.schedule(sub)
            for kind in ("content", "reference"):
                content = W.invocation_content(9, sub.n, reference=(kind == "reference"))
                dec = sg.schedule(cfg_x, sub, content)
                out[kind] = evaluate(p, cw, sub, content, {"table": table["cfg"], "surrogate": dec["cfg"]},
                                     slack, lam, noise_seed=31)
    print("training loss by epoch", hist, "held-out rmse", rmse, "margin", margin)
    for kind, r in out.items():
        agree = float((r["table"]["cfg"] == r["surrogate"]["cfg"]).mean())
        print(kind, {k: (v["violations"], v["cost"]) for k, v in r.items()}, "agreement", agree)
    ref, con = out["reference"], out["content"]
    assert 0.0 < margin < 0.05
    # on reference content (where the table is exact) the surrogate must not
    # degrade the table's decisions: cost regret <= 1%, extra misses <= 0.5 points
    assert ref["surrogate"]["cost"] <= 1.01 * ref["table"]["cost"]
    assert ref["surrogate"]["violations"] <= ref["table"]["violations"] + 0.005
    # on varied content it must gain: far fewer missed targets than the content-blind table
    assert con["surrogate"]["violations"] < 0.5 * con["table"]["violations"]
    assert hist[-1] < hist[0]


def test_native_arrival_process_batches_what_arrived(L, world):
    """llama_sg_run_arrivals: every request's decision comes back after it
    arrived, in calls of at most max_batch requests that each took only
    requests already arrived; decreasing arrival times are refused."""
    import torch
    from paper_2102_01887_b300 import surrogate as S
    p, inv, cw = world
    n = 3000
    rng = np.random.default_rng(8)
    idx = rng.integers(0, inv.n, n)
    arrive = np.cumsum(rng.exponential(1e9 / 2e5, n)).astype(np.int64)  # 2e5 per second
    content = S.content_inputs(W.invocation_content(6, n))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    with L.Scheduler(p) as s, L.MLP(max_batch=1024) as net:
        net.set_params(M.pack(perturbed_params(41)).astype(np.float32))
        cfg_x = S.config_inputs(p, cw)
        with S.SurrogateScheduler(s, net, max_inv=256, max_pairs=1 << 20) as sg:
            done = sg.run_arrivals(cfg_x, content, dev(inv.dag[idx]), dev(inv.op_local[idx]),
                                   dev(inv.start_us[idx]), arrive, inv.now_us, max_batch=256)
            with pytest.raises(L.LlamaError):
                sg.run_arrivals(cfg_x, content, dev(inv.dag[idx]), dev(inv.op_local[idx]), dev(inv.start_us[idx]),
                                arrive[::-1].copy(), inv.now_us, max_batch=256)
    assert (done >= arrive).all()
    # a call's requests share its completion time: consecutive runs, each at most 256 long
    ends = np.flatnonzero(np.diff(done) != 0)
    sizes = np.diff(np.concatenate([[-1], ends, [n - 1]]))
    assert (np.diff(done) >= 0).all() and sizes.max() <= 256 and sizes.sum() == n
