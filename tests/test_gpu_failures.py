"""Failure detection without faulting the GPU.

* A bounded device wait whose partner never arrives gives up at the
  context's poll limit, the kernel returns, and the failure surfaces through
  the ticket (ans_wait) and the matrix (ans_matrix_view) as ERR_INTERNAL; the
  context keeps working afterwards, exactly.
* An allocator hook that fails makes the call return ERR_OOM before any work
  is queued (its outputs stay untouched) and the context recovers once the
  allocator does.
* ans_wait with a zero timeout on a batch still queued behind other work
  returns ERR_TIMEOUT, and a later wait completes it.
Every failure is made on the host side of the wait or the allocation; no test
faults, traps or hangs the GPU.
"""
import time

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


def _batch_is_exact(ans, ctx, w):
    out = torch.zeros((w.nwin, 9), dtype=torch.int64, device="cuda")
    mats, summ, tk = ctx.batch_submit(_dev(w.src), _dev(w.dst), w.offsets, ans.BATCH_MATRICES | ans.BATCH_SUM,
                                      out=out)
    ctx.wait(tk)
    exp_m, exp_q, exp_s = oracle.batch(w.src, w.dst, w.offsets)
    assert ans.quantities_from_tensor(out) == exp_q
    for m, e in zip(mats, exp_m):
        assert all(np.array_equal(a, b) for a, b in zip(m.to_numpy(), e))
        m.free()
    assert all(np.array_equal(a, b) for a, b in zip(summ.to_numpy(), exp_s))
    summ.free()


def test_expired_device_wait_is_reported_and_the_context_recovers(mods):
    ans, synth = mods
    ctx = ans.Context(0)
    try:
        ctx.set_wait_limit(1000)
        t0 = time.perf_counter()
        m, tk = ctx.probe_wait_expiry()
        assert ctx.wait_status(tk, 30.0) == ans.ERR_INTERNAL
        assert time.perf_counter() - t0 < 20.0  # 1000 polls end in well under a second
        with pytest.raises(ans.AnsError) as e:
            m.view()
        assert e.value.code == ans.ERR_INTERNAL
        with pytest.raises(ans.AnsError) as e:
            m.quantities()
        assert e.value.code == ans.ERR_INTERNAL
        m.free()
        # the probe's failure does not leak into later work
        _batch_is_exact(ans, ctx, synth.generate(2, sizes=[30000, 0, 9000, 70000]))
        ctx.set_wait_limit(0)  # back to the default
        _, tk = ctx.probe_wait_expiry(want_matrix=False)
        assert ctx.wait_status(tk, 60.0) == ans.ERR_INTERNAL  # the default limit (~1 s) also ends
        _batch_is_exact(ans, ctx, synth.generate(3, nwin=3))
    finally:
        ctx.close()


def test_failed_allocation_queues_nothing_and_recovers(mods):
    ans, synth = mods
    alloc = ans.TorchAllocator(0)
    ctx = ans.Context(0, allocator=alloc)
    try:
        small = synth.generate(2, sizes=[5000, 7000])
        _batch_is_exact(ans, ctx, small)
        big = synth.generate(2, sizes=[200000, 150000, 3])
        alloc.fail_after = alloc.calls + 1  # the next allocation fails
        out = torch.full((big.nwin, 9), -7, dtype=torch.int64, device="cuda")
        with pytest.raises(ans.AnsError) as e:
            ctx.batch_submit(_dev(big.src), _dev(big.dst), big.offsets, ans.BATCH_MATRICES | ans.BATCH_SUM,
                             out=out)
        assert e.value.code == ans.ERR_OOM
        torch.cuda.synchronize()
        assert bool((out == -7).all())  # nothing ran for the refused batch
        alloc.fail_after = None
        _batch_is_exact(ans, ctx, big)
        _batch_is_exact(ans, ctx, small)
    finally:
        ctx.close()
    assert not alloc.live  # every block went back through the free hook


def test_zero_timeout_wait_on_a_queued_batch(mods):
    ans, synth = mods
    ctx = ans.Context(0)
    try:
        w = synth.generate(2, sizes=[40000, 20000])
        src, dst = _dev(w.src), _dev(w.dst)
        out = torch.zeros((w.nwin, 9), dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        torch.cuda._sleep(2_000_000_000)  # ~1 s of device spinning ahead of the batch on this stream
        mats, summ, tk = ctx.batch_submit(src, dst, w.offsets, ans.BATCH_SUM, out=out)
        assert ctx.wait_status(tk, 0.0) == ans.ERR_TIMEOUT
        assert ctx.wait_status(tk, 60.0) == ans.OK
        assert ans.quantities_from_tensor(out) == oracle.batch(w.src, w.dst, w.offsets)[1]
        summ.free()
        assert ctx.wait_status(tk, 1.0) == ans.ERR_INVALID_ARG  # a finished ticket is gone
    finally:
        ctx.close()


class _FailOnce:
    """Allocator hooks over torch's caching allocator whose allocation
    number `fail_at` (and only that one) returns NULL."""

    def __init__(self, ans, device=0):
        self.calls = 0
        self.fail_at = None
        self.sizes = []
        self.live = {}

        def _alloc(nbytes, stream, user):
            self.calls += 1
            self.sizes.append(int(nbytes))
            if self.fail_at is not None and self.calls == self.fail_at:
                return None
            ptr = torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))
            self.live[ptr] = int(nbytes)
            return ptr

        def _free(ptr, stream, user):
            if ptr:
                self.live.pop(ptr, None)
                torch.cuda.caching_allocator_delete(ptr)

        self.alloc_fn = ans.ALLOC_FN(_alloc)
        self.free_fn = ans.FREE_FN(_free)


def test_windows_gather_falls_back_when_its_buffer_is_refused(mods):
    """ans_batch_submit_windows on the packet-sort paths gathers the windows
    into one buffer first; when that buffer's allocation fails, the windows
    are analysed in place on the other paths -- still exact -- and the next
    call, allocating again, gathers."""
    ans, synth = mods
    alloc = _FailOnce(ans)
    ctx = ans.Context(0, allocator=alloc)
    try:
        ctx.set_tuning(agg_path=3, sum_path=2)
        w = synth.generate(5, sizes=[3000, 0, 8193, 40000, 1, 20000], first_window=17)
        pin = (torch.from_numpy(w.src.view(np.int32)).pin_memory(), torch.from_numpy(w.dst.view(np.int32)).pin_memory())
        wins = [(pin[0][int(a):int(b)], pin[1][int(a):int(b)]) for a, b in zip(w.offsets[:-1], w.offsets[1:])]
        exp_m, exp_q, exp_s = oracle.batch(w.src, w.dst, w.offsets)
        gather_bytes = 8 * w.total  # at least: the windows' pairs
        for attempt in range(2):
            first = alloc.calls + 1
            alloc.fail_at = first if attempt == 0 else None  # the call's first allocation: the gather buffer
            out = torch.zeros((w.nwin, 9), dtype=torch.int64, device="cuda")
            mats, summ, tk = ctx.batch_submit_windows(wins, ans.BATCH_MATRICES | ans.BATCH_SUM, out=out)
            ctx.wait(tk)
            assert alloc.sizes[first - 1] >= gather_bytes  # that first allocation was the gather buffer
            assert ans.quantities_from_tensor(out) == exp_q
            for m, e in zip(mats, exp_m):
                assert all(np.array_equal(a, b) for a, b in zip(m.to_numpy(), e))
                m.free()
            assert all(np.array_equal(a, b) for a, b in zip(summ.to_numpy(), exp_s))
            summ.free()
    finally:
        ctx.close()
    assert not alloc.live
