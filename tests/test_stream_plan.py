"""Batch planning of the out-of-core ingest (host logic, no GPU)."""
import numpy as np

from paper_2510_14050_gb300 import stream


def test_plan_batches_covers_every_window_once_within_the_cap():
    sizes = np.array([5, 0, 7, 20, 3, 3, 0, 9, 1])
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    for cap in (1, 8, 10, 21, 100):
        plan = stream.plan_batches(offs, cap)
        assert plan[0][0] == 0 and plan[-1][1] == len(sizes)
        assert all(a[1] == b[0] for a, b in zip(plan, plan[1:]))
        for a, b in plan:
            n = int(offs[b] - offs[a])
            assert n <= cap or b - a == 1  # a larger window forms a batch alone
            if b < len(sizes):  # greedy: the next window would not have fit
                assert int(offs[b + 1] - offs[a]) > cap
    assert stream.plan_batches(np.zeros(1, np.uint64), 10) == []
