"""Column statistics of large time sums by hash groups (Table I: unique
destinations, max fan-in; Sec. IV-C: max destination packets).

A time sum that may hold 2^24 or more links sorts its links by the bijective
mix fmix32(dst) for two digit passes only; each of the 2^16 groups of equal
low 16 bits is then counted in a shared-memory table.  The tests check the
sum's DCSR and nine quantities element by element against the oracle on
every time-sum path that uses it, for

* ordinary traffic (every group fits its table),
* a group holding more distinct destinations than its table takes (the
  destinations are chosen by inverting the mix, so their mixes share the
  low 16 bits): the two remaining passes and the run count must finish the
  sort instead -- once with the group counted in one table, once with the
  group cut in parts that each fit but together do not,
* groups of more than 2^16 links (the heaviest destinations), cut in parts
  and merged,
* the one destination whose mix is the table's empty marker.
"""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")

M1, M2 = 0x85EBCA6B, 0xC2B2AE35


def _unxorshift(x, s):
    y = x.copy()
    for _ in range(32 // s + 1):
        y = x ^ (y >> np.uint64(s))
    return y


def _fmix32(h):
    h = np.array(h, dtype=np.uint64)  # a copy: the steps below work in place
    m = np.uint64(0xFFFFFFFF)
    h ^= h >> np.uint64(16)
    h = (h * np.uint64(M1)) & m
    h ^= h >> np.uint64(13)
    h = (h * np.uint64(M2)) & m
    h ^= h >> np.uint64(16)
    return h


def _unfmix32(h):
    """Inverse of MurmurHash3's 32-bit finalizer (each step is invertible)."""
    m = np.uint64(0xFFFFFFFF)
    x = np.asarray(h, dtype=np.uint64) & m
    x = _unxorshift(x, 16) & m
    x = (x * np.uint64(pow(M2, -1, 1 << 32))) & m
    x = _unxorshift(x, 13) & m
    x = (x * np.uint64(pow(M1, -1, 1 << 32))) & m
    x = _unxorshift(x, 16) & m
    return x


def test_inverse_mix_round_trips():
    rng = np.random.default_rng(0)
    x = rng.integers(0, 1 << 32, 100000, dtype=np.uint64)
    assert np.array_equal(_fmix32(_unfmix32(x)), x)
    assert np.array_equal(_unfmix32(_fmix32(x)), x)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _workload(overflow):
    from paper_2510_14050_gb300 import synth
    w = synth.generate(4, nwin=130)  # 130 x 2^17 packets: above the 2^24-link bound
    src, dst = w.src.copy(), w.dst.copy()
    rng = np.random.default_rng(7)
    # the destination whose mix is the empty marker, in a few windows
    special = np.uint32(_unfmix32(np.uint64(0xFFFFFFFF)))
    idx = rng.choice(len(dst), 500, replace=False)
    dst[idx] = special
    # 7000 distinct destinations in group 0 (mix & 0xffff == 0), in window 5
    crafted = _unfmix32(np.arange(1, 7001, dtype=np.uint64) << np.uint64(16)).astype(np.uint32)
    a = int(w.offsets[5])
    if overflow == "table":  # one link each: 7000 keys in the group's one table
        dst[a:a + len(crafted)] = crafted
        src[a:a + len(crafted)] = rng.integers(0, 1 << 32, len(crafted), dtype=np.uint64).astype(np.uint32)
    elif overflow == "parts":  # 20 links each, sources rising with the destination: parts of ~3300 keys
        n = 20 * len(crafted)
        dst[a:a + n] = np.repeat(crafted, 20)
        src[a:a + n] = (np.arange(n, dtype=np.uint64) * np.uint64(1000)).astype(np.uint32)
    return synth.Windows(src, dst, w.offsets)


@pytest.mark.gpu
@pytest.mark.parametrize("overflow", [None, "table", "parts"])
def test_sum_column_statistics_by_hash_groups(overflow):
    from paper_2510_14050_gb300 import ans
    w = _workload(overflow)
    exp_q = [oracle.window_quantities(*w.window(i)) for i in range(w.nwin)]
    exp_sum = oracle.traffic_matrix(w.src, w.dst)
    exp_sq = oracle.network_quantities(exp_sum)
    src, dst = _dev(w.src), _dev(w.dst)
    ctx = ans.Context(0)
    try:
        for paths in (dict(agg_path=3, sum_path=2), dict(agg_path=0, sum_path=2), dict(agg_path=0, sum_path=1),
                      dict(agg_path=0, sum_path=0)):
            ctx.set_tuning(**paths)
            out = torch.zeros((w.nwin, 9), dtype=torch.int64, device="cuda")
            _, summ, tk = ctx.batch_submit(src, dst, w.offsets, ans.BATCH_SUM, out=out)
            ctx.wait(tk)
            assert ans.quantities_from_tensor(out) == exp_q, paths
            for name, a, b in zip(exp_sum._fields, summ.to_numpy(), exp_sum):
                assert np.array_equal(a, b), f"{paths}: sum {name}"
            assert summ.quantities() == exp_sq, paths
            summ.free()
    finally:
        ctx.close()
