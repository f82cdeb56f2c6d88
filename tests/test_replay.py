"""Call dumps (.npy) and their bit-exact replay: on the CPU the dump's round
trip (every array back with its dtype and shape) and the oracle on the loaded
problem giving the dumped decisions; on the GPU, a dumped library call
replayed through the library and through the oracle."""
import numpy as np
import pytest

import oracle
from paper_2102_01887_b300 import replay as R
from paper_2102_01887_b300 import workloads as W

FIELDS = ("cfg", "lat", "cost", "slack", "flags")


@pytest.mark.parametrize("seed", [0, 5])
def test_dump_round_trip_and_oracle_replay(tmp_path, seed):
    p, inv = W.random_small(seed, max_cfg=10, n_inv=50)
    exp, _ = oracle.schedule(p, inv, mode=oracle.MODE_ALPHA, alpha=(2, 3))
    R.dump(str(tmp_path), p, inv, exp, mode=oracle.MODE_ALPHA, alpha=(2, 3))
    q, inv2, dec, meta = R.load(str(tmp_path))
    for name in R.PROBLEM_ARRAYS:
        a, b = getattr(p, name), getattr(q, name)
        assert (a is None) == (b is None), name
        if a is not None:
            assert a.dtype == b.dtype and np.array_equal(a, b), name
    for name in R.INV_ARRAYS:
        assert np.array_equal(getattr(inv, name), getattr(inv2, name))
    assert inv2.now_us == inv.now_us and meta["alpha"] == [2, 3]
    again, _ = oracle.schedule(q, inv2, mode=meta["mode"], alpha=tuple(meta["alpha"]))
    for k in FIELDS:
        assert np.array_equal(again[k], dec[k]), k


@pytest.mark.gpu
@pytest.mark.parametrize("method", [0, 1], ids=["scan", "staircase"])
def test_gpu_call_replays_bit_exactly(cuda_device, tmp_path, method):
    from paper_2102_01887_b300 import build, llama as L
    build.build()
    p, inv = W.medium(n_inv=20_000)
    with L.Scheduler(p, method=method) as s:
        got, rc = s.schedule(inv)
    R.dump(str(tmp_path), p, inv, got, method=method)
    again, rc2, same = R.replay(str(tmp_path))
    assert rc2 == rc and same
    q, inv2, dec, _ = R.load(str(tmp_path))
    exp, _ = oracle.schedule(q, inv2)
    for k in FIELDS:
        assert np.array_equal(exp[k], dec[k]), k
