"""Batches whose window offsets live in device memory (ans_batch_submit,
Sec. III-C batching planned on the GPU): results equal the oracle exactly,
with and without a batch capacity, on every aggregation and time-sum path;
offsets produced by earlier GPU work on the stream are honoured without a
host round trip; invalid offsets are reported through the ticket and the
matrices, and the context stays usable."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    from paper_2510_14050_gb300 import ans, synth
    ans.load()
    return ans, synth


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _doffs(offsets, shift=0):
    return torch.from_numpy((np.asarray(offsets, dtype=np.uint64) + np.uint64(shift)).view(np.int64)).cuda()


def _check(ans, mats, summ, q, w, src=None, dst=None):
    src = w.src if src is None else src
    dst = w.dst if dst is None else dst
    exp_m, exp_q, exp_s = oracle.batch(src, dst, w.offsets)
    assert ans.quantities_from_tensor(q) == exp_q
    if mats is not None:
        for i, (m, e) in enumerate(zip(mats, exp_m)):
            for name, a, b in zip(e._fields, m.to_numpy(), e):
                assert np.array_equal(a, b), f"window {i}: {name}"
            assert m.quantities() == exp_q[i]
    for name, a, b in zip(exp_s._fields, summ.to_numpy(), exp_s):
        assert np.array_equal(a, b), f"sum: {name}"
    assert summ.quantities() == oracle.network_quantities(exp_s)


@pytest.mark.parametrize("cap", [0, 1 << 22])
@pytest.mark.parametrize("paths", [dict(sum_path=0, agg_path=0), dict(sum_path=1, agg_path=0),
                                   dict(sum_path=2, agg_path=0), dict(sum_path=0, agg_path=1),
                                   dict(sum_path=2, agg_path=1), dict(sum_path=2, agg_path=3),
                                   dict(sum_path=0, agg_path=3)])
def test_device_offsets_match_the_oracle(mods, cap, paths):
    ans, synth = mods
    sizes = synth.window_sizes(5, 14)
    sizes[[0, 6, 13]] = 0
    sizes[2] = 1
    sizes[9] = 8192
    sizes[10] = 8193
    w = synth.generate(5, sizes=sizes)
    # the windows start 100 packets into the arrays: offsets[0] != 0
    pad = 100
    src = _dev(np.concatenate([np.zeros(pad, np.uint32), w.src]))
    dst = _dev(np.concatenate([np.zeros(pad, np.uint32), w.dst]))
    ctx = ans.Context(0)
    try:
        ctx.set_tuning(**paths)
        ctx.set_batch_capacity(cap)
        for _ in range(2):  # the second call replays the cached graph
            q = torch.zeros((w.nwin, 9), dtype=torch.int64, device="cuda")
            mats, summ, tk = ctx.batch_submit(src, dst, _doffs(w.offsets, pad), ans.BATCH_MATRICES | ans.BATCH_SUM,
                                              out=q)
            ctx.wait(tk)
            _check(ans, mats, summ, q, w)
            # matrices of a device-planned batch in a later time sum and analysis
            again = ctx.sum_windows(mats[3:] + mats[:3])
            for a, b in zip(again.to_numpy(), summ.to_numpy()):
                assert np.array_equal(a, b)
            assert ctx.network_quantities(mats[4]) == mats[4].quantities()
            for m in mats:
                m.free()
            summ.free()
            again.free()
    finally:
        ctx.close()


def test_offsets_written_by_earlier_gpu_work(mods):
    """The offsets are computed on the device right before the call (a
    cumulative sum of window lengths on the same stream); the call reads
    them only on the device."""
    ans, synth = mods
    w = synth.generate(2, nwin=16)
    lens = torch.from_numpy(np.diff(w.offsets).astype(np.int64)).cuda()
    src, dst = _dev(w.src), _dev(w.dst)
    ctx = ans.Context(0)
    try:
        ctx.set_batch_capacity(w.total + 12345)
        for shuffle in (False, True):
            if shuffle:  # a different split of the same packets: the same capacity, other windows
                cut = np.sort(np.random.default_rng(1).choice(np.arange(1, w.total), 15, replace=False))
                w = synth.Windows(w.src, w.dst, np.concatenate([[0], cut, [w.total]]).astype(np.uint64))
                lens = torch.from_numpy(np.diff(w.offsets).astype(np.int64)).cuda()
            offs = torch.zeros(w.nwin + 1, dtype=torch.int64, device="cuda")
            torch.cumsum(lens, 0, out=offs[1:])
            q = torch.zeros((w.nwin, 9), dtype=torch.int64, device="cuda")
            _, summ, tk = ctx.batch_submit(src, dst, offs, ans.BATCH_SUM, out=q)
            ctx.wait(tk)
            _check(ans, None, summ, q, w)
            summ.free()
    finally:
        ctx.close()


@pytest.mark.parametrize("bad", ["decreasing", "over_capacity"])
def test_invalid_device_offsets_are_reported(mods, bad):
    ans, synth = mods
    w = synth.generate(2, sizes=[3000, 4000, 5000])
    offs = np.asarray(w.offsets, dtype=np.uint64).copy()
    ctx = ans.Context(0)
    try:
        if bad == "decreasing":
            offs[1], offs[2] = offs[2], offs[1]
            ctx.set_batch_capacity(w.total)
        else:
            ctx.set_batch_capacity(w.total - 1)
        q = torch.full((w.nwin, 9), -1, dtype=torch.int64, device="cuda")
        mats, summ, tk = ctx.batch_submit(_dev(w.src), _dev(w.dst), _doffs(offs), ans.BATCH_MATRICES | ans.BATCH_SUM,
                                          out=q)
        assert ctx.wait_status(tk, 60.0) == ans.ERR_INVALID_ARG
        with pytest.raises(ans.AnsError) as e:
            mats[0].view()
        assert e.value.code == ans.ERR_INVALID_ARG
        with pytest.raises(ans.AnsError) as e:
            summ.quantities()
        assert e.value.code == ans.ERR_INVALID_ARG
        assert bool((q == 0).all())  # every window came out empty
        for m in mats:
            m.free()
        summ.free()
        # the context keeps working
        ctx.set_batch_capacity(0)
        q = torch.zeros((w.nwin, 9), dtype=torch.int64, device="cuda")
        mats, summ, tk = ctx.batch_submit(_dev(w.src), _dev(w.dst), _doffs(w.offsets),
                                          ans.BATCH_MATRICES | ans.BATCH_SUM, out=q)
        ctx.wait(tk)
        _check(ans, mats, summ, q, w)
    finally:
        ctx.close()
