"""Stragglers and failed invocations (Section 3.4; the 1.5x time-out of
Section 5): which invocations get a duplicate and when it is handed back.
Host code of the library (llama_stragglers), checked on hand-derived cases;
no GPU is used."""
import numpy as np
import pytest

from paper_2102_01887_b300 import llama as L


@pytest.fixture(scope="module")
def lib():
    from paper_2102_01887_b300 import build
    build.build()
    return L.load()


def decisions(cfg, lat):
    d = np.zeros(len(cfg), L.DECISION_DTYPE)
    d["cfg"], d["lat"] = cfg, lat
    return d


def test_time_out_is_three_halves_of_the_latency_rounded_up(lib):
    # latency 100: time-out at 150 us; 101: ceil(151.5) = 152
    d = decisions([0, 0, 0, 0], [100, 100, 101, 101])
    idx, when = L.llama_stragglers(d, [150, 151, 152, 153], None, 1000)
    assert idx.tolist() == [1, 3]             # ran past its time-out
    assert when.tolist() == [1150, 1152]      # handed back at the time-out itself


def test_errors_before_the_time_out_give_a_duplicate_when_they_arrive(lib):
    d = decisions([2, 2, 2, -1], [100, 100, 100, 100])
    failed = [1, 1, 0, 1]
    # an error at 40 us; an error that would come at 400 us is preceded by the
    # time-out at 150; a clean completion; an undecided invocation (nothing ran)
    idx, when = L.llama_stragglers(d, [40, 400, 120, 10], failed, 5000)
    assert idx.tolist() == [0, 1]
    assert when.tolist() == [5040, 5150]


def test_hand_back_at_the_managers_next_tick(lib):
    d = decisions([1, 1, 1], [1000, 1000, 1000])
    # events at now + 10, + 1500 (time-out), + 1000 (error); ticks of 1,000 us
    idx, when = L.llama_stragglers(d, [10, 5000, 1000], [1, 0, 1], 20_000, tick_us=1000)
    assert idx.tolist() == [0, 1, 2]
    assert when.tolist() == [21_000, 22_000, 21_000]


def test_other_time_out_factors_and_nothing_to_do(lib):
    d = decisions([0, 0], [10, 10])
    idx, _ = L.llama_stragglers(d, [20, 21], None, 0, timeout=(2, 1))
    assert idx.tolist() == [1]
    idx, when = L.llama_stragglers(d[:0], [], None, 0)
    assert idx.size == 0 and when.size == 0


def test_bad_arguments(lib):
    d = decisions([0], [10])
    for kw in ({"timeout": (0, 1)}, {"timeout": (1, 0)}, {"tick_us": 0}):
        with pytest.raises(L.LlamaError):
            L.llama_stragglers(d, [5], None, 0, **kw)
    with pytest.raises(L.LlamaError):
        L.llama_stragglers(d, [-1], None, 0)  # negative observed time
