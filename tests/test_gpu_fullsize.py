"""GPU parity at full size: the mixed 1024-window workload (~1.5 x 10^8
packets) and the 2^30-packet workload (8192 windows of 2^17 packets over the
full 2^32 address space), element by element against the oracle.

For each workload:
* the batch as the bench runs it (autotuned paths, per-window quantities +
  the time sum): every window's nine quantities, and the whole time-summed
  DCSR -- checked row slice by row slice against the oracle's matrix of the
  packets whose sources fall in the slice -- with the sum's quantities;
* the same batch on other (aggregation, time-sum) paths -- on the
  1024-window workload every time-sum path with the window sort and the
  windows from the packet sort, on the 2^30-packet workload the window sort
  with merge rounds (and the windows from the packet sort, unless tuned) --
  the last with per-window matrices: their time sums again, and the DCSR of
  every window (1024-window workload) or of 130 windows (2^30-packet
  workload).
Tolerance 0: every output is an integer with one correct value.
"""
import numpy as np
import pytest

from tests import fullsize

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SLICES = {3: 64, 4: 256}


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _run(ans, ctx, src, dst, w, flags):
    out = torch.zeros((w.nwin, 9), dtype=torch.int64, device="cuda")
    mats, summ, tk = ctx.batch_submit(src, dst, w.offsets, flags, out=out)
    ctx.wait(tk)
    return mats, summ, ans.quantities_from_tensor(out)


@pytest.mark.parametrize("cfg", [3, 4])
def test_full_size_batch_against_oracle(cfg):
    from paper_2510_14050_gb300 import ans, synth
    w = synth.generate(cfg)
    src, dst = _dev(w.src), _dev(w.dst)
    results = []  # host copies of the GPU time sums
    ctx = ans.Context(0)
    try:
        tuned = ctx.autotune(src, dst, w.offsets, flags=ans.BATCH_SUM)
        _, summ, q = _run(ans, ctx, src, dst, w, ans.BATCH_SUM)
        mine = (tuned["agg_path"], 2 if tuned["agg_path"] == 3 else tuned["sum_path"])
        results.append((f"bench paths (agg_path {mine[0]}, sum_path {mine[1]})", summ.to_numpy(), summ.quantities()))
        summ.free()
        # other (aggregation, time-sum) paths, the last with per-window matrices
        if cfg == 3:
            others = [x for x in [(0, 0), (0, 1), (0, 2), (3, 2)] if x != mine]
        else:
            others = [x for x in [(3, 2), (0, 0)] if x != mine]
        for k, (ap, sp) in enumerate(others):
            ctx.set_tuning(agg_path=ap, sum_path=sp)
            last = k == len(others) - 1
            mats, summ2, q2 = _run(ans, ctx, src, dst, w, ans.BATCH_SUM | (ans.BATCH_MATRICES if last else 0))
            results.append((f"agg_path {ap}, sum_path {sp}", summ2.to_numpy(), summ2.quantities()))
            summ2.free()
            assert q2 == q
        rng = np.random.default_rng(cfg)
        ids = list(range(w.nwin)) if cfg == 3 else sorted(
            set(rng.choice(w.nwin, 128, replace=False).tolist()) | {0, w.nwin - 1})
        got = {i: mats[i].to_numpy() for i in ids}
        quants = {i: mats[i].quantities() for i in ids}
        for m in mats:
            m.free()
    finally:
        ctx.close()
    del src, dst
    torch.cuda.empty_cache()

    # every window's quantities
    exp_q = fullsize.window_quantities(w)
    for i in range(w.nwin):
        assert q[i] == exp_q[i], f"window {i} quantities"
    # whole-window DCSR
    exp_m = fullsize.window_matrices(w, ids)
    for i, e in zip(ids, exp_m):
        for name, a, b in zip(e._fields, got[i], e):
            assert np.array_equal(a, b), f"window {i}: {name}"
        assert quants[i] == exp_q[i]
    # the time sums, row slice by row slice, and their quantities
    bad, exp_sq = fullsize.check_time_sum(w.src, w.dst, [r[1] for r in results], SLICES[cfg])
    assert not bad, f"time sum differs from the oracle: {bad[:5]} ({[r[0] for r in results]})"
    assert exp_sq["valid_packets"] == w.total
    for what, _, sq in results:
        assert sq == exp_sq, what
