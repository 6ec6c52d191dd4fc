"""The full-size slice check of the time sum (tests/fullsize.py), pinned on
a batch small enough for the oracle's plain time sum: it must agree with it,
and it must find a planted difference.  No GPU needed."""
import numpy as np

import oracle
from tests import fullsize


def test_row_slices_pin_the_sum_on_a_small_batch():
    """The slice check itself, against the oracle's plain time sum on a batch
    small enough for it, with a planted difference it must find."""
    from paper_2510_14050_gb300 import synth
    w = synth.generate(3, nwin=24, first_window=7)
    exp_m, _, exp_sum = oracle.batch(w.src, w.dst, w.offsets)
    gpu_like = tuple(np.array(a) for a in exp_sum)
    bad, q = fullsize.check_time_sum(w.src, w.dst, [gpu_like], 16)
    assert not bad and q == oracle.network_quantities(exp_sum)
    wrong = tuple(np.array(a) for a in exp_sum)
    wrong[3][len(wrong[3]) // 2] += np.uint64(1)
    bad, _ = fullsize.check_time_sum(w.src, w.dst, [wrong], 16)
    assert bad and bad[0][3] == "vals"


def test_row_slices_cover_every_row():
    from paper_2510_14050_gb300 import synth
    w = synth.generate(4, nwin=3)
    s = oracle.traffic_matrix(w.src, w.dst)
    edges = [fullsize.SPACE * i // 8 for i in range(9)]
    parts = [fullsize.rows_of(tuple(s), a, b) for a, b in zip(edges[:-1], edges[1:])]
    assert sum(p.nrows for p in parts) == s.nrows and sum(p.nnz for p in parts) == s.nnz
    assert np.array_equal(np.concatenate([p.col_ids for p in parts]), s.col_ids)
