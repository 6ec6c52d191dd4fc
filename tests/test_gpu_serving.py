"""Serving: continuous batching gives every window the same result alone and
in the mix (tolerance 0), and the resident tumbling time sums equal the
oracle's sum of the windows in each bucket."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _alone(ctx, src, dst):
    m = ctx.build_window(_dev(src if len(src) else [0]), _dev(dst if len(dst) else [0]), len(src))
    q = m.quantities()
    m.free()
    return q


@pytest.mark.parametrize("slots,budget,zero_copy", [(3, 48 << 30, True), (2, 3 << 30, True), (2, 3 << 30, False)])
def test_alone_equals_mix_and_bucket_sums(slots, budget, zero_copy):
    from paper_2510_14050_gb300 import ans, serve, synth
    pool = 24
    src = serve.pool_source(pool, seed=3)
    n = 72
    arrivals = np.sort(synth.arrivals(4000.0, n, seed=5))
    order = (np.arange(n) * 5) % pool
    srv = serve.Server(device=0, slots=slots, budget_bytes=budget, max_batch_windows=7,
                       max_batch_packets=1 << 21, bucket_seconds=(0.005, 0.02), zero_copy=zero_copy)
    try:
        stats = srv.serve(src, arrivals, order)
        assert stats.batches >= 2
        assert len(stats.latencies_s) == n and np.all(stats.latencies_s > 0)
        ctx = ans.Context(0)
        alone = {}
        for w in range(pool):
            a, b = int(src.offsets[w]), int(src.offsets[w + 1])
            alone[w] = _alone(ctx, src.src[a:b], src.dst[a:b])
            assert alone[w] == oracle.window_quantities(src.src[a:b], src.dst[a:b])
        ctx.close()
        for k in range(n):
            got = dict(zip(oracle.QUANTITY_NAMES, (int(v) for v in stats.quantities[k])))
            assert got == alone[int(order[k])], f"arrival {k}"
        # resident tumbling sums: compare every bucket of both levels with the oracle
        for level, width in enumerate(srv.bucket_seconds):
            ids = (arrivals // width).astype(int)
            for idx in np.unique(ids):
                ks = np.nonzero(ids == idx)[0]
                mats = []
                for k in ks:
                    w = int(order[k])
                    a, b = int(src.offsets[w]), int(src.offsets[w + 1])
                    mats.append(oracle.traffic_matrix(src.src[a:b], src.dst[a:b]))
                exp = oracle.sum_matrices(mats)
                got = srv.bucket_sum(level, int(idx))
                assert got is not None
                for x, y in zip(got.to_numpy(), exp):
                    assert np.array_equal(x, y), f"bucket {level}/{idx}"
                assert got.quantities() == oracle.network_quantities(exp)
    finally:
        srv.close()


def test_small_budget_stalls_admission_but_stays_exact():
    from paper_2510_14050_gb300 import ans, serve, synth
    pool = 8
    src = serve.pool_source(pool, seed=9)
    n = 24
    arrivals = np.zeros(n)  # everything arrives at once
    order = np.full(n, 3)   # equal batches: each needs the same working set
    # The budget fits one slot's working set, not two: the second slot is
    # refused admission while the first one runs.
    probe = ans.Context(0)
    one = np.concatenate([[0], np.cumsum([src.size(3)] * 4)]).astype(np.uint64)
    need = probe.batch_bytes(one, 0)
    probe.close()
    srv = serve.Server(device=0, slots=2, budget_bytes=int(need * 1.5), max_batch_windows=4,
                       max_batch_packets=1 << 20, bucket_seconds=(60.0,), keep_sums=False)
    try:
        stats = srv.serve(src, arrivals, order)
        assert stats.batches >= n // 4
        assert stats.admission_stalls > 0
        assert srv.live_bytes() <= srv.budget
        for k in range(n):
            w = int(order[k])
            a, b = int(src.offsets[w]), int(src.offsets[w + 1])
            exp = oracle.window_quantities(src.src[a:b], src.dst[a:b])
            assert dict(zip(oracle.QUANTITY_NAMES, (int(v) for v in stats.quantities[k]))) == exp
    finally:
        srv.close()


def test_sliding_sum_and_checkpoint_restore(tmp_path):
    """A 40 ms sliding sum in 10 ms steps equals the oracle's sum of the
    windows whose step lies in the newest four steps (the older ones were
    added and later subtracted); the resident sums survive a checkpoint and a
    restore into a fresh server bit for bit."""
    from paper_2510_14050_gb300 import serve, synth
    pool = 16
    src = serve.pool_source(pool, seed=11)
    n = 60
    arrivals = np.sort(synth.arrivals(500.0, n, seed=13))  # about 0.12 s of arrivals
    order = (np.arange(n) * 3) % pool
    step, horizon = 0.01, 0.04
    kw = dict(device=0, slots=2, budget_bytes=48 << 30, max_batch_windows=5, max_batch_packets=1 << 21,
              bucket_seconds=(0.05,), sliding=((horizon, step),))
    srv = serve.Server(**kw)
    try:
        stats = srv.serve(src, arrivals, order)
        assert stats.batches >= 4
        sub = (arrivals // step).astype(int)
        last = sub.max()
        ks = np.nonzero(sub > last - int(round(horizon / step)))[0]
        mats = []
        for k in ks:
            w = int(order[k])
            a, b = int(src.offsets[w]), int(src.offsets[w + 1])
            mats.append(oracle.traffic_matrix(src.src[a:b], src.dst[a:b]))
        exp = oracle.sum_matrices(mats)
        got = srv.sliding_sum(0)
        for x, y in zip(got.to_numpy(), exp):
            assert np.array_equal(x, y)
        assert got.quantities() == oracle.network_quantities(exp)
        got.free()
        ids = (arrivals // 0.05).astype(int)
        before = {int(i): [a.copy() for a in srv.bucket_sum(0, int(i)).to_numpy()] for i in np.unique(ids)}
        path = tmp_path / "sums.npz"
        srv.checkpoint(str(path))
    finally:
        srv.close()
    again = serve.Server(**kw)
    try:
        again.restore(str(path))
        for i, arrays in before.items():
            for x, y in zip(again.bucket_sum(0, i).to_numpy(), arrays):
                assert np.array_equal(x, y)
        got = again.sliding_sum(0)
        for x, y in zip(got.to_numpy(), exp):
            assert np.array_equal(x, y)
        got.free()
    finally:
        again.close()
