"""Scratch guards: a debug mode standing in for a memory checker.

A context created with ANS_SCRATCH_GUARDS=1 puts 256 bytes of a fixed
pattern after every region of a batch's scratch layout and of its output
blocks, writes them before the batch's kernels and compares them after; an
overwritten guard makes the batch report ERR_INTERNAL.

* ans_probe_guards overwrites a guard's first word, as a write one word past
  its region would, and the check must report it (the context stays usable);
* batches on every aggregation and time-sum path, with and without
  per-window matrices, host and device offsets, windows in their own arrays,
  at ragged sizes around the 8192-item tile (empty, one packet, 8191, 8193,
  more than 2^17 packets), leave every guard intact and equal the oracle.
Nothing here writes outside an allocation: the probe's write lands inside
the guard, which is part of the scratch arena.
"""
import os

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = [0, 1, 8191, 8193, 40000, 0, 131072, 150001, 3]


@pytest.fixture(scope="module")
def mods():
    from paper_2510_14050_gb300 import ans, synth
    ans.load()
    return ans, synth


@pytest.fixture()
def guarded(mods):
    ans, _ = mods
    old = os.environ.get("ANS_SCRATCH_GUARDS")
    os.environ["ANS_SCRATCH_GUARDS"] = "1"
    try:
        ctx = ans.Context(0)
    finally:
        if old is None:
            del os.environ["ANS_SCRATCH_GUARDS"]
        else:
            os.environ["ANS_SCRATCH_GUARDS"] = old
    yield ctx
    ctx.close()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _check(ans, ctx, w, flags, offsets=None, windows=False, expected=None):
    out = torch.zeros((max(w.nwin, 1), 9), dtype=torch.int64, device="cuda")
    if windows:
        wins = [(_dev(w.src[a:b]), _dev(w.dst[a:b])) for a, b in zip(w.offsets[:-1], w.offsets[1:])]
        mats, summ, tk = ctx.batch_submit_windows(wins, flags, out=out)
    else:
        mats, summ, tk = ctx.batch_submit(_dev(w.src), _dev(w.dst), w.offsets if offsets is None else offsets,
                                          flags, out=out)
    assert ctx.wait_status(tk) == ans.OK, ans.status_string(ctx.wait_status(tk))
    exp_m, exp_q, exp_s = expected or oracle.batch(w.src, w.dst, w.offsets, want_sum=bool(flags & ans.BATCH_SUM))
    assert ans.quantities_from_tensor(out)[: w.nwin] == exp_q
    for m, e in zip(mats or [], exp_m):
        assert all(np.array_equal(a, b) for a, b in zip(m.to_numpy(), e))
        m.free()
    if summ is not None:
        assert all(np.array_equal(a, b) for a, b in zip(summ.to_numpy(), exp_s))
        summ.free()


def test_probe_reports_an_overwritten_guard(mods, guarded):
    ans, synth = mods
    tk = guarded.probe_guards()
    assert guarded.wait_status(tk) == ans.ERR_INTERNAL
    # the context keeps working, guards and all
    _check(ans, guarded, synth.generate(5, sizes=[3000, 8193]), ans.BATCH_MATRICES | ans.BATCH_SUM)


@pytest.mark.parametrize("agg_path,sum_path", [(0, 0), (0, 1), (0, 2), (1, 0), (2, 2), (3, 2)])
def test_batches_leave_every_guard_intact(mods, guarded, agg_path, sum_path):
    ans, synth = mods
    guarded.set_tuning(agg_path=agg_path, sum_path=sum_path)
    w = synth.generate(5, sizes=SIZES, first_window=agg_path * 10 + sum_path)
    for flags in (ans.BATCH_MATRICES | ans.BATCH_SUM, ans.BATCH_SUM, ans.BATCH_MATRICES):
        _check(ans, guarded, w, flags)
    _check(ans, guarded, w, ans.BATCH_MATRICES | ans.BATCH_SUM,
           offsets=torch.from_numpy(w.offsets.astype(np.int64)).cuda())
    _check(ans, guarded, w, ans.BATCH_MATRICES | ans.BATCH_SUM, windows=True)


def test_guards_on_the_large_workload_shapes(mods, guarded):
    """Windows of the 1024-window and 2^30-packet workloads' kinds (a heavy
    hitter and scanners; 2^32-wide Zipf addresses), through the column
    hash's destination partitions and -- 136 windows of 2^17 packets, a time
    sum above 2^24 links -- the time sum's hash groups."""
    ans, synth = mods
    for cfg, nwin in ((3, 24), (4, 136)):
        w = synth.generate(cfg, nwin=nwin)
        expected = oracle.batch(w.src, w.dst, w.offsets)
        for ap in (0, 3):
            guarded.set_tuning(agg_path=ap, sum_path=2)
            _check(ans, guarded, w, ans.BATCH_SUM, expected=expected)
