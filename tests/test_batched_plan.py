"""Host logic of the batched solver: the worker assignment of
gbhe_batched_plan (no GPU needed)."""
import numpy as np
import pytest

from paper_1207_1773_gb300 import gbhegv


def test_plan_is_deterministic_and_balanced():
    rng = np.random.default_rng(3)
    ns = [int(v) for v in rng.integers(500, 3001, 64)]
    a1 = gbhegv.batched_plan(ns, 8)
    a2 = gbhegv.batched_plan(ns, 8)
    assert a1 == a2
    assert set(a1) == set(range(8))
    load = np.zeros(8)
    for n, k in zip(ns, a1):
        load[k] += float(n) ** 3
    # greedy largest-first: no worker exceeds another by more than the largest job
    assert load.max() - load.min() <= max(ns) ** 3


def test_plan_largest_first_and_edge_cases():
    assert gbhegv.batched_plan([10, 30, 20], 1) == [0, 0, 0]
    # the largest problem goes to worker 0, the next to worker 1, ...
    assert gbhegv.batched_plan([10, 30, 20], 3) == [2, 0, 1]
    assert gbhegv.batched_plan([], 4) == []
    with pytest.raises(gbhegv.GbheError):
        gbhegv.batched_plan([5], 0)
    with pytest.raises(gbhegv.GbheError):
        gbhegv.batched_plan([-1], 2)
