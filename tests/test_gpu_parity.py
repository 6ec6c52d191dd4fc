"""GPU parity: every result of the CUDA path equals the oracle bit for bit.

All inputs are seeded and synthetic; every call goes through the C ABI
(libans.so) via the ctypes binding.  Tolerance is zero: the outputs are
integers (DCSR structure, uint64 counts, the nine quantities) and exactly one
canonical answer exists.
"""
import numpy as np
import pytest

import oracle
from tests import golden_io

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KT = 8192  # tile size of the kernels: sizes around multiples of it are edge cases


@pytest.fixture(scope="module")
def ans():
    from paper_2510_14050_gb300 import ans as mod
    mod.load()
    return mod


@pytest.fixture(scope="module")
def ctx(ans):
    c = ans.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def synth():
    from paper_2510_14050_gb300 import synth as mod
    return mod


def dev(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint32))
    return torch.from_numpy(a.view(np.int32)).cuda()


def assert_dcsr_equal(got, exp: oracle.DCSR, what=""):
    r, p, c, v = got
    assert np.array_equal(r, exp.row_ids), f"{what}: row_ids differ"
    assert np.array_equal(p, exp.row_ptr), f"{what}: row_ptr differ"
    assert np.array_equal(c, exp.col_ids), f"{what}: col_ids differ"
    assert np.array_equal(v, exp.vals), f"{what}: vals differ"


def check_window(ctx, src, dst, what=""):
    m = ctx.build_window(dev(src), dev(dst), len(src))
    exp = oracle.traffic_matrix(src, dst)
    assert_dcsr_equal(m.to_numpy(), exp, what)
    q = oracle.network_quantities(exp)
    assert m.quantities() == q, what
    assert ctx.network_quantities(m) == q, what
    return m


@pytest.mark.parametrize("name", golden_io.FIXTURES)
def test_golden_windows(ctx, name):
    (win,), exp = golden_io.load(name)
    m = ctx.build_window(dev(win[0]), dev(win[1]), len(win[0]))
    r, p, c, v = m.to_numpy()
    assert [int(x) for x in r] == exp["row_ids"] and [int(x) for x in p] == exp["row_ptr"]
    assert [int(x) for x in c] == exp["col_ids"] and [int(x) for x in v] == exp["vals"]
    assert m.quantities() == {k: exp[k][0] for k in oracle.QUANTITY_NAMES}


def test_golden_time_sum(ctx):
    wins, exp = golden_io.load("time_sum.txt")
    mats = [ctx.build_window(dev(s), dev(d), len(s)) for s, d in wins]
    s = ctx.sum_windows(mats)
    r, p, c, v = s.to_numpy()
    assert [int(x) for x in r] == exp["sum_row_ids"] and [int(x) for x in p] == exp["sum_row_ptr"]
    assert [int(x) for x in c] == exp["sum_col_ids"] and [int(x) for x in v] == exp["sum_vals"]
    q = {k: exp["sum_" + k][0] for k in oracle.QUANTITY_NAMES}
    assert s.quantities() == q
    assert ctx.network_quantities(s) == q


def test_empty_and_single(ctx):
    m = ctx.build_window(dev([0]), dev([0]), 0)
    assert m.view()[:2] == (0, 0)
    r, p, c, v = m.to_numpy()
    assert list(p) == [0]
    assert m.quantities() == dict.fromkeys(oracle.QUANTITY_NAMES, 0)
    assert ctx.network_quantities(m) == dict.fromkeys(oracle.QUANTITY_NAMES, 0)
    check_window(ctx, np.array([0xFFFFFFFF], np.uint32), np.array([0xFFFFFFFF], np.uint32), "single max key")
    check_window(ctx, np.array([0], np.uint32), np.array([0], np.uint32), "single zero key")


@pytest.mark.parametrize("n", [KT - 1, KT, KT + 1, 2 * KT + 7, 5 * KT + 1])
def test_identical_packets_span_tiles(ctx, n):
    check_window(ctx, np.full(n, 0xFFFFFFFF, np.uint32), np.full(n, 0xFFFFFFFF, np.uint32), f"identical {n}")
    check_window(ctx, np.full(n, 9, np.uint32), np.zeros(n, np.uint32), f"identical0 {n}")


@pytest.mark.parametrize("n", [1, 31, 33, 511, 513, KT - 1, KT, KT + 1, 3 * KT - 5, 40000])
def test_random_ragged_sizes(ctx, n):
    rng = np.random.default_rng(n)
    pool = rng.integers(0, 2**32, size=max(2, n // 5), dtype=np.uint64).astype(np.uint32)
    pool[0], pool[-1] = 0, 0xFFFFFFFF
    src = pool[rng.integers(0, len(pool), n)]
    dst = pool[rng.integers(0, len(pool), n)]
    check_window(ctx, src, dst, f"random {n}")


def test_distinct_star_and_reverse_star(ctx):
    rng = np.random.default_rng(5)
    p = 3 * KT + 11
    src = (rng.permutation(p).astype(np.uint64) * 2654435761 % 2**32).astype(np.uint32)
    dst = rng.permutation(p).astype(np.uint32)
    check_window(ctx, src, dst, "distinct")
    star_d = (np.arange(2 * KT + 3, dtype=np.uint64) * 40503 % 2**32).astype(np.uint32)
    star_s = np.full(len(star_d), 77, np.uint32)
    check_window(ctx, star_s, star_d, "star")
    check_window(ctx, star_d, star_s, "reverse star")


@pytest.mark.parametrize("shift", [1, 2, 3])
def test_unaligned_inputs(ctx, shift):
    rng = np.random.default_rng(shift)
    n = 2 * KT + 100
    src = rng.integers(0, 300, n + shift).astype(np.uint32)
    dst = rng.integers(0, 300, n + shift).astype(np.uint32)
    ds, dd = dev(src), dev(dst)
    m = ctx.build_window(ds[shift:], dd[shift:], n)
    exp = oracle.traffic_matrix(src[shift:], dst[shift:])
    assert_dcsr_equal(m.to_numpy(), exp, "unaligned")
    assert m.quantities() == oracle.network_quantities(exp)


def test_cfg1_single_window(ctx, synth):
    w = synth.generate(1)
    check_window(ctx, w.src, w.dst, "cfg1")


def run_batch(ans, ctx, w, flags):
    out = torch.zeros((w.nwin, 9), dtype=torch.int64, device="cuda")
    mats, summ, tk = ctx.batch_submit(dev(w.src), dev(w.dst), w.offsets, flags, out=out)
    ctx.wait(tk)
    return mats, summ, ans.quantities_from_tensor(out)


def check_batch(ans, ctx, w, check_mats=True, check_sum=True):
    flags = (ans.BATCH_MATRICES if check_mats else 0) | (ans.BATCH_SUM if check_sum else 0)
    mats, summ, quants = run_batch(ans, ctx, w, flags)
    exp_mats, exp_q, exp_sum = oracle.batch(w.src, w.dst, w.offsets, want_sum=check_sum)
    for i in range(w.nwin):
        assert quants[i] == exp_q[i], f"window {i}"
        if check_mats:
            assert_dcsr_equal(mats[i].to_numpy(), exp_mats[i], f"window {i}")
            assert mats[i].quantities() == exp_q[i]
    if check_sum:
        assert_dcsr_equal(summ.to_numpy(), exp_sum, "sum")
        sq = oracle.network_quantities(exp_sum)
        assert summ.quantities() == sq
        assert ctx.network_quantities(summ) == sq
    return mats, summ, quants


def test_batch_cfg2_full(ans, ctx, synth):
    w = synth.generate(2)
    check_batch(ans, ctx, w)


def test_batch_cfg3_subset(ans, ctx, synth):
    w = synth.generate(3, nwin=48)
    check_batch(ans, ctx, w)


def test_batch_cfg4_subset(ans, ctx, synth):
    w = synth.generate(4, nwin=12)
    check_batch(ans, ctx, w)


def test_batch_cfg5_with_empty_windows(ans, ctx, synth):
    sizes = synth.window_sizes(5, 20)
    sizes[[0, 7, 19]] = 0
    sizes[3] = 1
    sizes[11] = KT
    w = synth.generate(5, sizes=sizes)
    check_batch(ans, ctx, w)


def test_empty_batch(ans, ctx):
    mats, summ, tk = ctx.batch_submit(dev([0]), dev([0]), np.zeros(1, np.uint64),
                                      ans.BATCH_MATRICES | ans.BATCH_SUM)
    ctx.wait(tk)
    assert mats == [] and summ.view()[:2] == (0, 0)
    assert summ.quantities() == dict.fromkeys(oracle.QUANTITY_NAMES, 0)


def test_batched_equals_per_window_and_sum_across_calls(ans, ctx, synth):
    w = synth.generate(5, nwin=6)
    mats, summ, quants = run_batch(ans, ctx, w, ans.BATCH_MATRICES | ans.BATCH_SUM)
    singles = []
    for i in range(w.nwin):
        s, d = w.window(i)
        m = ctx.build_window(dev(s), dev(d), len(s))
        for a, b in zip(m.to_numpy(), mats[i].to_numpy()):
            assert np.array_equal(a, b)
        assert m.quantities() == quants[i]
        singles.append(m)
    # a time sum over matrices that came from different calls
    mixed = ctx.sum_windows(singles[:3] + mats[3:])
    for a, b in zip(mixed.to_numpy(), summ.to_numpy()):
        assert np.array_equal(a, b)
    # summing sums: (A0 + A1) + (A2 + ... ) == total
    part1 = ctx.sum_windows(mats[:2])
    part2 = ctx.sum_windows(singles[2:])
    total = ctx.sum_windows([part1, part2])
    for a, b in zip(total.to_numpy(), summ.to_numpy()):
        assert np.array_equal(a, b)


def test_quantities_only_batch_matches(ans, ctx, synth):
    w = synth.generate(3, nwin=20, first_window=100)
    _, _, quants = run_batch(ans, ctx, w, 0)
    exp = [oracle.window_quantities(*w.window(i)) for i in range(w.nwin)]
    assert quants == exp


def test_memory_budget_refuses_and_recovers(ans, synth):
    w = synth.generate(2, nwin=8)
    c = ans.Context(0, budget_bytes=64 << 20)
    try:
        with pytest.raises(ans.AnsError) as ei:
            c.batch_submit(dev(w.src), dev(w.dst), w.offsets, ans.BATCH_MATRICES)
        assert ei.value.code == ans.ERR_BUDGET
        s, d = w.window(0)
        small = 5000
        m = c.build_window(dev(s[:small]), dev(d[:small]), small)
        assert m.quantities() == oracle.window_quantities(s[:small], d[:small])
        m.free()
    finally:
        c.close()


def test_invalid_arguments(ans, ctx):
    with pytest.raises(ans.AnsError) as ei:
        ctx.batch_submit(dev([1, 2]), dev([1, 2]), np.array([0, 2, 1], np.uint64), 0)
    assert ei.value.code == ans.ERR_INVALID_ARG
    with pytest.raises(ans.AnsError) as ei:
        ctx.wait(123456789)
    assert ei.value.code == ans.ERR_INVALID_ARG


@pytest.mark.parametrize("threads,rank,blocks", [(512, 0, 1), (512, 1, 1), (512, 2, 1), (512, 0, 2), (512, 1, 2),
                                                 (512, 2, 2), (1024, 0, 1), (1024, 1, 1), (1024, 2, 1)])
def test_every_sort_configuration_is_exact(ans, synth, threads, rank, blocks):
    """Results never depend on the radix-pass launch configuration."""
    w = synth.generate(5, sizes=[KT * 3 + 17, 0, 40000, 1, 2 * KT])
    c = ans.Context(0)
    try:
        c.set_tuning(key_threads=threads, key_rank=rank, key_blocks=blocks, kv_threads=threads, kv_rank=rank,
                     kv_blocks=blocks, col_threads=threads, col_rank=rank, col_blocks=blocks, win_path=1)
        assert c.get_tuning()["kv_threads"] == threads
        check_batch(ans, c, w)
    finally:
        c.close()


@pytest.mark.parametrize("rank", [0, 1, 2])
def test_key_passes_over_subtiles_are_exact(ans, synth, rank):
    """Key and column passes that split every tile into two 4096-key
    sub-tiles give the same results: windows ending inside either half of a
    tile, exactly at the half, one key past it, empty and single-packet
    windows, windows the column hash leaves to the column sort, the time sum,
    and the one-window path."""
    h = KT // 2
    w = synth.generate(5, sizes=[KT * 3 + 17, 0, h, h + 1, h - 1, 1, 2 * KT, KT + h, 40000])
    src, dst = w.src.copy(), w.dst.copy()
    a, b = int(w.offsets[8]), int(w.offsets[9])
    dst[a:b] = np.random.default_rng(rank).integers(0, 1 << 32, b - a, dtype=np.uint64).astype(np.uint32)
    from paper_2510_14050_gb300 import synth as sy
    w = sy.Windows(src, dst, w.offsets)
    c = ans.Context(0)
    try:
        c.set_tuning(key_threads=256, key_rank=rank, key_blocks=4, col_threads=256, col_rank=rank, col_blocks=4,
                     win_path=1)
        assert c.get_tuning()["key_threads"] == 256 and c.get_tuning()["col_threads"] == 256
        check_batch(ans, c, w)
        check_window(c, *w.window(8), "one window").free()
        for bad in ({"key_threads": 256, "key_blocks": 2}, {"kv_threads": 256, "kv_blocks": 4},
                    {"col_threads": 256, "col_blocks": 2}):
            with pytest.raises(ans.AnsError) as ei:
                c.set_tuning(**bad)
            assert ei.value.code == ans.ERR_INVALID_ARG
    finally:
        c.close()


def test_autotune_picks_valid_configuration(ans, synth):
    w = synth.generate(2, nwin=4)
    c = ans.Context(0)
    try:
        t = c.autotune(dev(w.src), dev(w.dst), w.offsets)
        assert t["key_threads"] in (256, 512, 1024) and t["col_rank"] in (0, 1, 2) and t["key_rank"] in (0, 1, 2)
        assert c.get_tuning() == t
        check_batch(ans, c, w)
        with pytest.raises(ans.AnsError) as ei:
            c.set_tuning(key_threads=384)
        assert ei.value.code == ans.ERR_INVALID_ARG
    finally:
        c.close()


# Windows sorted on chip by one 8-CTA cluster (at most 2^17 packets, spread
# over the CTAs in power-of-two slices of 512 .. 16384 keys) next to windows
# that take the onesweep passes, in one batch.
CLUSTER_SIZES = [0, 1, 511, 512, 513, 4095, 4097, 16383, 16384, 16385, 65539, 131071, 131072, 131073, 200000]


@pytest.mark.parametrize("path,threads,rank", [(0, 1024, 0), (0, 1024, 1), (0, 512, 0), (0, 512, 1), (1, 1024, 0)])
def test_window_sort_paths_are_exact(ans, synth, path, threads, rank):
    w = synth.generate(5, sizes=CLUSTER_SIZES)
    c = ans.Context(0)
    try:
        c.set_tuning(win_path=path, win_threads=threads, win_rank=rank)
        assert c.get_tuning()["win_path"] == path
        check_batch(ans, c, w)
    finally:
        c.close()


@pytest.mark.parametrize("path", [0, 1])
@pytest.mark.parametrize("n", [1 << 17, (1 << 17) - 1])
def test_window_sort_degenerate_windows(ans, n, path):
    """Every key equal (one digit in every pass), and one source to n distinct
    destinations (all keys share the upper four digits), on both window
    paths."""
    c = ans.Context(0)
    try:
        c.set_tuning(win_path=path)
        z = np.full(n, 0xDEADBEEF, np.uint32)
        check_window(c, z, z, "identical").free()
        rng = np.random.default_rng(n)
        d = rng.permutation(np.arange(n, dtype=np.uint64) * 7919 % (1 << 32)).astype(np.uint32)
        check_window(c, np.full(n, 5, np.uint32), d, "star").free()
        check_window(c, d, np.full(n, 0xFFFFFFFF, np.uint32), "reverse star").free()
    finally:
        c.close()


@pytest.mark.parametrize("sum_path,merge_tile", [(0, 4096), (0, 2048), (1, 4096), (2, 4096)])
@pytest.mark.parametrize("nwin", [1, 2, 3, 5, 8, 13])
def test_time_sum_paths_are_exact(ans, synth, sum_path, merge_tile, nwin):
    """Time sums by pairwise merges (0, with either merge tile), by radix
    passes over the windows' links (1) and by sorting the batch's packets
    again (2), for window counts that leave odd runs and empty windows at
    every merge round."""
    sizes = [(i * 7919) % 30000 if i % 4 != 2 else 0 for i in range(nwin)]
    sizes[0] = max(sizes[0], 3)
    w = synth.generate(5, sizes=sizes, first_window=nwin)
    c = ans.Context(0)
    try:
        c.set_tuning(sum_path=sum_path, merge_tile=merge_tile)
        with pytest.raises(ans.AnsError):
            c.set_tuning(merge_tile=1024)
        mats, summ, _ = check_batch(ans, c, w)
        # sums of sums and of matrices in another order
        exp = oracle.sum_matrices([oracle.traffic_matrix(*w.window(i)) for i in range(nwin)])
        half = c.sum_windows(mats[::2])
        rest = c.sum_windows(mats[1::2]) if nwin > 1 else None
        total = c.sum_windows([half, rest] if rest is not None else [half])
        assert_dcsr_equal(total.to_numpy(), exp, "sum of sums")
        rev = c.sum_windows(mats[::-1])
        assert_dcsr_equal(rev.to_numpy(), exp, "reversed")
    finally:
        c.close()


def test_matrices_outlive_their_context(ans, synth):
    """A matrix stays readable after ans_ctx_destroy; the last matrix freed
    releases the context's remaining state."""
    w = synth.generate(5, sizes=[5000, 7000])
    c = ans.Context(0)
    mats, summ, _ = c.batch_submit(dev(w.src), dev(w.dst), w.offsets, ans.BATCH_MATRICES | ans.BATCH_SUM,
                                   want_ticket=False)
    single = c.build_window(dev(w.window(0)[0]), dev(w.window(0)[1]), 5000)
    c.close()
    for i, m in enumerate(mats):
        exp = oracle.traffic_matrix(*w.window(i))
        assert_dcsr_equal(m.to_numpy(), exp, f"window {i}")
        assert m.quantities() == oracle.network_quantities(exp)
        m.free()
    assert_dcsr_equal(summ.to_numpy(), oracle.sum_matrices([oracle.traffic_matrix(*w.window(i)) for i in range(2)]))
    summ.free()
    assert_dcsr_equal(single.to_numpy(), oracle.traffic_matrix(*w.window(0)))
    single.free()


def _dup_heavy_window(n, links, seed):
    """n packets drawn from `links` distinct (src, dst) pairs, the all-ones
    pair (the hash tables' empty marker) among them."""
    rng = np.random.default_rng(seed)
    s = rng.integers(0, 1 << 32, links, dtype=np.uint64).astype(np.uint32)
    d = rng.integers(0, 1 << 32, links, dtype=np.uint64).astype(np.uint32)
    s[0] = d[0] = 0xFFFFFFFF
    pick = rng.integers(0, links, n)
    return s[pick], d[pick]


@pytest.mark.parametrize("agg_path", [0, 1])
def test_aggregation_paths_are_exact(ans, synth, agg_path):
    """Sorting every packet (0) and hash counting then sorting the distinct
    links (1) give the same DCSR and quantities: mixed window sizes (empty,
    ragged, larger than 2^17), heavy duplication with the all-ones key, all
    packets equal, all distinct."""
    w = synth.generate(5, sizes=[0, 1, 8191, 8193, 40000, 0, 131072, 150001], first_window=7)
    c = ans.Context(0)
    try:
        c.set_tuning(agg_path=agg_path)
        assert c.get_tuning()["agg_path"] == agg_path
        for _ in range(2):  # the second call reuses the (emptied) tables
            check_batch(ans, c, w)
        for n, links in [(100000, 37), (65536, 1), (20000, 20000)]:
            s, d = _dup_heavy_window(n, links, n + links)
            check_window(c, s, d, f"{n}/{links}").free()
        z = np.full(50000, 0xFFFFFFFF, np.uint32)
        check_window(c, z, z, "all ones").free()
        perm = np.random.default_rng(1).permutation(1 << 16).astype(np.uint32)
        check_window(c, perm, perm[::-1].copy(), "distinct").free()
        w3 = synth.generate(3, nwin=6, first_window=40)
        check_batch(ans, c, w3)
    finally:
        c.close()


@pytest.mark.parametrize("sum_path", [0, 2])
def test_windows_from_the_packet_sort(ans, synth, sum_path):
    """agg_path 3: the windows' sorted keys come from the time sum's packet
    sort (the packets carry their window ids; a stable two-pass sort by
    window id puts every window back at its base).  Exact against the oracle
    with and without per-window matrices, whatever sum_path says: mixed
    sizes (empty, one packet, ragged tiles, larger than 2^17), more than 256
    windows (both id digits), exactly 2^16 windows (the largest id), and the
    batches the path leaves to the window sort (one window, 2^16 + 1 windows,
    no time sum)."""
    c = ans.Context(0)
    try:
        c.set_tuning(agg_path=3, sum_path=sum_path)
        assert c.get_tuning()["agg_path"] == 3
        w = synth.generate(5, sizes=[0, 1, 8191, 8193, 40000, 0, 131072, 150001], first_window=7)
        for _ in range(2):  # the second call replays the cached graph
            check_batch(ans, c, w)
        check_batch(ans, c, w, check_mats=False)
        rng = np.random.default_rng(5)
        sizes = rng.integers(0, 3000, 700)
        sizes[[0, 255, 256, 511, 699]] = [0, 1, 8192, 0, 5]
        check_batch(ans, c, synth.generate(5, sizes=sizes, first_window=3))
        check_batch(ans, c, synth.generate(3, nwin=6, first_window=40))
        for nwin in (1 << 16, (1 << 16) + 1):
            sizes = rng.integers(0, 4, nwin)
            sizes[-1] = 2
            check_batch(ans, c, synth.generate(5, sizes=sizes, first_window=1), check_mats=False)
        check_batch(ans, c, synth.generate(5, sizes=[5000]))              # one window
        check_batch(ans, c, synth.generate(5, nwin=4), check_sum=False)  # no time sum
    finally:
        c.close()


@pytest.mark.parametrize("agg_path", [0, 1, 2, 3])
def test_pairs_read_in_place_from_pinned_host_memory(ans, synth, agg_path):
    """The packet arrays given as page-locked host memory: the kernels read
    them in place over the host link.  Exact against the oracle on every
    aggregation path, with host and device offsets, with the arrays at an
    offset that breaks 16-byte alignment, and equal to the same batch from
    device copies of the arrays."""
    c = ans.Context(0)
    try:
        c.set_tuning(agg_path=agg_path, sum_path=2 if agg_path >= 2 else 0)
        w = synth.generate(5, sizes=[0, 1, 8191, 8193, 40000, 0, 131072], first_window=21)
        one = np.ones(1, dtype=np.uint32)
        src_h = torch.from_numpy(np.concatenate([7 * one, w.src]).view(np.int32))
        dst_h = torch.from_numpy(np.concatenate([9 * one, w.dst]).view(np.int32))
        assert src_h.numel() == w.total + 1 and dst_h.numel() == w.total + 1
        src_h, dst_h = src_h.pin_memory(), dst_h.pin_memory()
        offs = w.offsets + 1  # the first pair of each array is not part of the batch
        exp_mats, exp_q, exp_sum = oracle.batch(w.src, w.dst, w.offsets)
        for offsets in (offs, torch.from_numpy(offs.astype(np.int64)).cuda()):
            for flags in (ans.BATCH_MATRICES | ans.BATCH_SUM, ans.BATCH_SUM):
                out = torch.zeros((w.nwin, 9), dtype=torch.int64, device="cuda")
                mats, summ, tk = c.batch_submit(src_h, dst_h, offsets, flags, out=out)
                c.wait(tk)
                assert ans.quantities_from_tensor(out) == exp_q
                for i, m in enumerate(mats or []):
                    assert_dcsr_equal(m.to_numpy(), exp_mats[i], f"window {i}")
                    m.free()
                assert_dcsr_equal(summ.to_numpy(), exp_sum, "sum")
                assert summ.quantities() == oracle.network_quantities(exp_sum)
                summ.free()
    finally:
        c.close()


@pytest.mark.parametrize("agg_path,sum_path", [(0, 0), (3, 2), (2, 2), (0, 2)])
def test_windows_in_their_own_arrays(ans, synth, agg_path, sum_path):
    """ans_batch_submit_windows with every window in its own arrays -- in
    page-locked host memory at word offsets of every alignment modulo 16, or
    in device memory -- exact against the oracle on each path; on the paths
    that sort the batch's packets as one segment a kernel first gathers the
    windows into one device buffer (the copy's vector and word forms, window
    lengths around the 1024-word vector chunk and the tile)."""
    c = ans.Context(0)
    try:
        c.set_tuning(agg_path=agg_path, sum_path=sum_path)
        w = synth.generate(5, sizes=[0, 1, 3, 1023, 1025, 8191, 8193, 40000, 0, 131072], first_window=31)
        pool_src = torch.from_numpy(np.concatenate([np.arange(64, dtype=np.uint32), w.src]).view(np.int32))
        pool_dst = torch.from_numpy(np.concatenate([np.arange(64, dtype=np.uint32), w.dst]).view(np.int32))
        pin_src, pin_dst = pool_src.pin_memory(), pool_dst.pin_memory()
        dev_src, dev_dst = pool_src.cuda(), pool_dst.cuda()
        exp_mats, exp_q, exp_sum = oracle.batch(w.src, w.dst, w.offsets)
        for where in ("pinned", "device"):
            s_all, d_all = (pin_src, pin_dst) if where == "pinned" else (dev_src, dev_dst)
            wins = []
            for i in range(w.nwin):
                a, b = int(w.offsets[i]), int(w.offsets[i + 1])
                # window i's copy starts `shift` words further into a shifted copy of the pool
                shift = i % 4
                base_s = s_all.data_ptr() + 4 * (64 + a)
                base_d = d_all.data_ptr() + 4 * (64 + a)
                if shift:  # the same pairs, read from a copy placed `shift` words later
                    cs = torch.empty(b - a + shift, dtype=torch.int32)
                    cd = torch.empty(b - a + shift, dtype=torch.int32)
                    cs[shift:] = torch.from_numpy(w.src[a:b].view(np.int32))
                    cd[shift:] = torch.from_numpy(w.dst[a:b].view(np.int32))
                    cs, cd = (cs.pin_memory(), cd.pin_memory()) if where == "pinned" else (cs.cuda(), cd.cuda())
                    wins.append((cs, cd))  # keep the copies alive
                    base_s, base_d = cs.data_ptr() + 4 * shift, cd.data_ptr() + 4 * shift
                wins.append((base_s, base_d, b - a))
            triples = [x for x in wins if len(x) == 3]
            for flags in (ans.BATCH_MATRICES | ans.BATCH_SUM, ans.BATCH_SUM):
                out = torch.zeros((w.nwin, 9), dtype=torch.int64, device="cuda")
                mats, summ, tk = c.batch_submit_windows(triples, flags, out=out)
                c.wait(tk)
                assert ans.quantities_from_tensor(out) == exp_q, where
                for i, m in enumerate(mats or []):
                    assert_dcsr_equal(m.to_numpy(), exp_mats[i], f"{where} window {i}")
                    m.free()
                assert_dcsr_equal(summ.to_numpy(), exp_sum, f"{where} sum")
                summ.free()
    finally:
        c.close()


@pytest.mark.parametrize("graph", [0, 1])
def test_graph_replay_follows_each_call(ans, synth, graph):
    """With graph replay, a cached executable graph is reused for batches of
    the same shape: each call's own inputs and outputs must be the ones used
    (new device buffers, different packets, same shape), across shape
    changes and back."""
    a1 = synth.generate(5, sizes=[3000, 0, 20000, 8192], first_window=1)
    a2 = synth.generate(5, sizes=[3000, 0, 20000, 8192], first_window=11)  # same shape, other packets
    b = synth.generate(2, nwin=5, first_window=3)
    c = ans.Context(0)
    try:
        c.set_tuning(graph=graph)
        for w in (a1, b, a2, a1, a2, b, a1):
            check_batch(ans, c, w)
        # quantities-only calls of the same windows, into caller-owned outputs
        for w in (a2, a1):
            _, _, quants = run_batch(ans, c, w, 0)
            assert quants == [oracle.window_quantities(*w.window(i)) for i in range(w.nwin)]
    finally:
        c.close()


def test_import_dcsr_quantities_and_sums(ans, ctx, synth):
    """Matrices given as DCSR (the paper's input form) get the oracle's
    quantities, read back unchanged, and sum with built windows."""
    w = synth.generate(2, nwin=3, first_window=50)
    exp = [oracle.traffic_matrix(*w.window(i)) for i in range(3)]
    imported = []
    for i, e in enumerate(exp):
        if i == 0:  # host arrays
            m = ctx.import_matrix(e.row_ids, e.row_ptr, e.col_ids, e.vals)
        else:       # device tensors
            t = [torch.from_numpy(np.ascontiguousarray(a).view(np.int32 if a.dtype == np.uint32 else np.int64)).cuda()
                 for a in (e.row_ids, e.row_ptr, e.col_ids, e.vals)]
            m = ctx.import_matrix(*t)
        assert_dcsr_equal(m.to_numpy(), e, f"import {i}")
        assert m.quantities() == oracle.network_quantities(e)
        assert ctx.network_quantities(m) == oracle.network_quantities(e)
        imported.append(m)
    built = ctx.build_window(dev(w.window(2)[0]), dev(w.window(2)[1]), int(w.offsets[3] - w.offsets[2]))
    s = ctx.sum_windows(imported[:2] + [built])
    assert_dcsr_equal(s.to_numpy(), oracle.sum_matrices(exp), "sum")
    for m in imported + [built, s]:
        m.free()
    empty = ctx.import_matrix(np.zeros(0, np.uint32), np.zeros(1, np.uint64), np.zeros(0, np.uint32),
                              np.zeros(0, np.uint64))
    assert empty.quantities() == dict.fromkeys(oracle.QUANTITY_NAMES, 0)
    empty.free()


@pytest.mark.parametrize("case", ["row_ptr_start", "empty_row", "rows_unsorted", "zero_value", "cols_unsorted",
                                  "cols_equal", "row_ptr_end"])
def test_import_rejects_non_canonical_dcsr(ans, ctx, case):
    r = np.array([1, 5, 9], np.uint32)
    p = np.array([0, 2, 3, 5], np.uint64)
    c = np.array([3, 7, 2, 0, 4], np.uint32)
    v = np.array([1, 2, 3, 4, 5], np.uint64)
    m = ctx.import_matrix(r, p, c, v)  # canonical: accepted
    m.free()
    r, p, c, v = r.copy(), p.copy(), c.copy(), v.copy()
    if case == "row_ptr_start":
        p[0] = 1
    elif case == "empty_row":
        p[1] = 0
    elif case == "rows_unsorted":
        r[1], r[2] = 9, 5
    elif case == "zero_value":
        v[3] = 0
    elif case == "cols_unsorted":
        c[0], c[1] = 7, 3
    elif case == "cols_equal":
        c[4] = 0
    elif case == "row_ptr_end":
        p[3] = 4
    with pytest.raises(ans.AnsError) as ei:
        ctx.import_matrix(r, p, c, v)
    assert ei.value.code == ans.ERR_INVALID_ARG


@pytest.mark.parametrize("where", ["device", "pinned", "mixed"])
def test_batch_of_scattered_windows(ans, ctx, synth, where):
    """Windows in their own arrays -- device tensors, pinned host tensors read
    in place by the kernels, or both in one batch -- give the oracle's
    matrices, quantities and time sum; unaligned starts and empty windows
    included."""
    w = synth.generate(5, sizes=[40000, 0, 8193, 131072, 3, 200001], first_window=77)
    wins = []
    for i in range(w.nwin):
        s, d = w.window(i)
        pad = i % 3  # start some windows off a 16-byte boundary
        st = torch.from_numpy(np.concatenate([np.zeros(pad, np.uint32), s]).view(np.int32))[pad:]
        dt = torch.from_numpy(np.concatenate([np.zeros(pad, np.uint32), d]).view(np.int32))[pad:]
        on_dev = where == "device" or (where == "mixed" and i % 2 == 0)
        if on_dev:
            st, dt = st.cuda(), dt.cuda()
        else:
            base_s = torch.zeros(len(s) + pad, dtype=torch.int32).pin_memory()
            base_d = torch.zeros(len(d) + pad, dtype=torch.int32).pin_memory()
            base_s[pad:] = st
            base_d[pad:] = dt
            st, dt = base_s[pad:], base_d[pad:]
        wins.append((st, dt))
    out = torch.zeros((w.nwin, 9), dtype=torch.int64, device="cuda")
    mats, summ, tk = ctx.batch_submit_windows(wins, ans.BATCH_MATRICES | ans.BATCH_SUM, out=out)
    ctx.wait(tk)
    exp_mats, exp_q, exp_sum = oracle.batch(w.src, w.dst, w.offsets, want_sum=True)
    got_q = ans.quantities_from_tensor(out)
    for i in range(w.nwin):
        assert got_q[i] == exp_q[i], f"window {i}"
        assert_dcsr_equal(mats[i].to_numpy(), exp_mats[i], f"window {i}")
        mats[i].free()
    assert_dcsr_equal(summ.to_numpy(), exp_sum, "sum")
    summ.free()


def test_signed_combination_subtracts_exactly(ans, ctx, synth):
    """A sliding-sum update: (A + B + C) - B = A + C exactly, with the links
    only B had dropped rather than stored as zeros; all-positive signs equal
    ans_sum_windows; a count driven negative is reported."""
    w = synth.generate(2, nwin=3, first_window=300)
    ms = [ctx.build_window(dev(w.window(i)[0]), dev(w.window(i)[1]), int(w.offsets[i + 1] - w.offsets[i]))
          for i in range(3)]
    exp = [oracle.traffic_matrix(*w.window(i)) for i in range(3)]
    total = ctx.combine(ms, [1, 1, 1])
    assert_dcsr_equal(total.to_numpy(), oracle.sum_matrices(exp), "sum")
    same = ctx.sum_windows(ms)
    assert_dcsr_equal(same.to_numpy(), oracle.sum_matrices(exp), "sum_windows")
    slid = ctx.combine([total, ms[1]], [1, -1])
    want = oracle.sum_matrices([exp[0], exp[2]])
    assert_dcsr_equal(slid.to_numpy(), want, "after subtraction")
    assert slid.quantities() == oracle.network_quantities(want)
    assert ctx.network_quantities(slid) == oracle.network_quantities(want)
    # everything leaves: the empty matrix
    gone = ctx.combine([slid, ms[0], ms[2]], [1, -1, -1])
    assert gone.view()[:2] == (0, 0)
    assert gone.quantities() == dict.fromkeys(oracle.QUANTITY_NAMES, 0)
    # more taken out than was in
    bad = ctx.combine([ms[0], ms[1]], [1, -1])
    with pytest.raises(ans.AnsError) as ei:
        bad.quantities()
    assert ei.value.code == ans.ERR_INVALID_ARG
    for m in ms + [total, same, slid, gone, bad]:
        m.free()
    with pytest.raises(ans.AnsError) as ei:
        ctx.combine([ctx.build_window(dev([1]), dev([2]), 1)], [0])
    assert ei.value.code == ans.ERR_INVALID_ARG


@pytest.mark.parametrize("col_hash", [0, 1])
def test_column_statistics_by_hash_or_sort(ans, synth, col_hash):
    """Window column statistics from the shared-memory destination hash (and
    the sort for windows whose destinations overflow it) equal the oracle:
    few and many distinct destinations, the all-ones destination, fan-in
    concentrated on one destination, and more destinations than the table
    holds."""
    rng = np.random.default_rng(5)
    sizes = [0, 1, 5000, 131072, 30000, 70000]
    w = synth.generate(5, sizes=sizes, first_window=123)
    src, dst = w.src.copy(), w.dst.copy()
    a, b = int(w.offsets[4]), int(w.offsets[5])
    dst[a:b:3] = 0xFFFFFFFF  # the empty-slot marker as a real destination, heavily
    a, b = int(w.offsets[5]), int(w.offsets[6])
    dst[a:b] = rng.integers(0, 1 << 32, b - a, dtype=np.uint64).astype(np.uint32)  # > 12288 destinations
    from paper_2510_14050_gb300 import synth as sy
    w2 = sy.Windows(src, dst, w.offsets)
    c = ans.Context(0)
    try:
        c.set_tuning(col_hash=col_hash)
        check_batch(ans, c, w2)
    finally:
        c.close()


@pytest.mark.parametrize("nwin", [1, 3, 20, 40, 80])
def test_column_hash_over_clusters(ans, nwin):
    """Window column statistics when several CTAs share a window's hash (as
    many as the batch leaves SMs for: 8, 4, 2 or 1 per window): windows with
    exactly the table's limit of distinct destinations (12288), one more,
    more in total than the limit while every CTA's share stays below it, the
    all-ones destination, few destinations, and empty and one-packet
    windows, all equal to the oracle."""
    from paper_2510_14050_gb300 import synth as sy
    rng = np.random.default_rng(nwin)
    wins = []
    for i in range(nwin):
        kind = i % 7
        if kind == 0:
            d = np.repeat(rng.permutation(1 << 20)[:12288].astype(np.uint32), 3)
        elif kind == 1:
            d = np.repeat(rng.permutation(1 << 20)[:12289].astype(np.uint32), 2)
        elif kind == 2:
            d = rng.permutation(1 << 20)[:20000].astype(np.uint32)
        elif kind == 3:
            d = rng.integers(0, 50, 30000).astype(np.uint32)
            d[::4] = 0xFFFFFFFF
        elif kind == 4:
            d = np.zeros(0, np.uint32)
        elif kind == 5:
            d = np.array([7], np.uint32)
        else:
            d = rng.integers(0, 5000, 60000).astype(np.uint32)
        rng.shuffle(d)
        wins.append((rng.integers(0, 1 << 12, len(d)).astype(np.uint32), d))
    offsets = np.zeros(nwin + 1, np.uint64)
    offsets[1:] = np.cumsum([len(d) for _, d in wins])
    w = sy.Windows(np.concatenate([s_ for s_, _ in wins]), np.concatenate([d for _, d in wins]), offsets)
    c = ans.Context(0)
    try:
        check_batch(ans, c, w, check_sum=nwin <= 20)
    finally:
        c.close()


def _fmix32(h):
    """MurmurHash3's 32-bit finalizer (Appleby), vectorised."""
    h = np.asarray(h, dtype=np.uint64)
    m = np.uint64(0xFFFFFFFF)
    h ^= h >> np.uint64(16)
    h = (h * np.uint64(0x85EBCA6B)) & m
    h ^= h >> np.uint64(13)
    h = (h * np.uint64(0xC2B2AE35)) & m
    h ^= h >> np.uint64(16)
    return h


@pytest.mark.parametrize("col_hash", [1, 0])
def test_column_hash_over_destination_partitions(ans, col_hash):
    """Windows with more distinct destinations than one shared-memory table
    holds: split into 2..32 destination partitions (8192 links each) by the
    partitioned hash, with the boundaries of its range (2^18 links, one more),
    windows whose links hit few destinations, the all-ones destination among
    many, and a window whose destinations all fall in one partition (it
    overflows its table and is left to the column sort) -- all equal to the
    oracle, whichever path each window takes."""
    from paper_2510_14050_gb300 import synth as sy
    rng = np.random.default_rng(17)
    wins = []
    for n in (8193, 16384, 16385, 60000, 150000, 1 << 18, (1 << 18) + 1):
        d = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
        if n == 60000:
            d[::5] = 0xFFFFFFFF
        wins.append((rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32), d))
    # few destinations behind many links: the one-table hash finishes it
    wins.append((rng.integers(0, 1 << 32, 100000, dtype=np.uint64).astype(np.uint32),
                 rng.integers(0, 3000, 100000).astype(np.uint32)))
    # 16000 distinct destinations, all in partition 0 of 2: that table overflows
    cand = rng.integers(0, 1 << 32, 200000, dtype=np.uint64).astype(np.uint32)
    part = ((_fmix32(cand) >> np.uint64(14)) * np.uint64(2)) >> np.uint64(18)
    d = np.unique(cand[part == 0])[:16000]
    assert len(d) == 16000
    wins.append((rng.integers(0, 1 << 32, len(d), dtype=np.uint64).astype(np.uint32), rng.permutation(d)))
    offsets = np.zeros(len(wins) + 1, np.uint64)
    offsets[1:] = np.cumsum([len(x) for x, _ in wins])
    w = sy.Windows(np.concatenate([x for x, _ in wins]), np.concatenate([y for _, y in wins]), offsets)
    c = ans.Context(0)
    try:
        c.set_tuning(col_hash=col_hash)
        check_batch(ans, c, w, check_sum=False)
        _, _, quants = run_batch(ans, c, w, 0)  # quantities only: the DCSR arrays stay in scratch
        assert quants == [oracle.window_quantities(*w.window(i)) for i in range(w.nwin)]
    finally:
        c.close()


def test_graph_cache_follows_column_hash_shape(ans, synth):
    """Batches whose window counts give the same merge depth but a different
    column-hash cluster shape (19 windows: 8 CTAs per window; 20 or 21: 4;
    38: 4; 39: 2) follow one another on one context, replayed as graphs;
    every result equals the oracle."""
    c = ans.Context(0)
    try:
        for i, nwin in enumerate([19, 20, 19, 21, 38, 39, 38]):
            w = synth.generate(5, sizes=synth.window_sizes(5, nwin, first_window=100 * i) // 16 + 1,
                               first_window=100 * i)
            _, summ, quants = run_batch(ans, c, w, ans.BATCH_SUM)
            _, exp_q, exp_sum = oracle.batch(w.src, w.dst, w.offsets, want_sum=True)
            assert quants == exp_q, f"batch {i} ({nwin} windows)"
            assert summ.quantities() == oracle.network_quantities(exp_sum), f"batch {i} sum"
            summ.free()
    finally:
        c.close()


def test_sum_column_statistics_across_calls(ans, synth):
    """One context sums batches that grow (its scratch is replaced), shrink,
    repeat, include the all-ones destination and a destination that takes
    most of the links, with the window column hash switched off and on
    again; every sum's quantities equal the oracle's."""
    rng = np.random.default_rng(11)
    c = ans.Context(0)
    try:
        for i, (nwin, col_hash) in enumerate([(3, 1), (40, 1), (2, 1), (2, 1), (9, 0), (9, 1)]):
            w = synth.generate(5, nwin=nwin, first_window=10 * i)
            dst = w.dst.copy()
            if i == 2:
                dst[::5] = 0xFFFFFFFF
            if i == 3:
                dst[rng.random(len(dst)) < 0.7] = 77
            c.set_tuning(col_hash=col_hash)
            _, summ, _ = run_batch(ans, c, synth.Windows(w.src, dst, w.offsets), ans.BATCH_SUM)
            exp = oracle.batch(w.src, dst, w.offsets, want_sum=True)[2]
            assert summ.quantities() == oracle.network_quantities(exp), f"call {i}"
            summ.free()
    finally:
        c.close()


def _fmix64(k):
    """MurmurHash3's 64-bit finalizer (Appleby), vectorised."""
    k = np.asarray(k, dtype=np.uint64).copy()
    k ^= k >> np.uint64(33)
    k *= np.uint64(0xFF51AFD7ED558CCD)
    k ^= k >> np.uint64(33)
    k *= np.uint64(0xC4CEB9FE1A85EC53)
    k ^= k >> np.uint64(33)
    return k


@pytest.mark.parametrize("with_sum", [False, True])
def test_hashed_window_statistics(ans, synth, with_sum):
    """Aggregation path 2 (every quantity by on-chip hashing, no sort) on
    windows of every workload's traffic, empty and one-packet windows, the
    all-ones link, source and destination, a window above its 2^18-packet
    limit, a window whose links all fall in one link partition (that table
    overflows) and one whose distinct sources all fall in one source
    partition (that table overflows): those windows are sorted instead, and
    every window equals the oracle; with a time sum (taken from the packets)."""
    from paper_2510_14050_gb300 import synth as sy
    rng = np.random.default_rng(5)
    wins = [synth.generate(4, nwin=3).window(i) for i in range(3)]
    wins += [synth.generate(2, nwin=2, first_window=9).window(i) for i in range(2)]
    w3 = synth.generate(3, nwin=6, first_window=40)
    wins += [w3.window(i) for i in range(6)]
    wins.append((np.zeros(0, np.uint32), np.zeros(0, np.uint32)))
    wins.append((np.array([0xFFFFFFFF], np.uint32), np.array([0xFFFFFFFF], np.uint32)))
    s = rng.integers(0, 1 << 32, 50000, dtype=np.uint64).astype(np.uint32)
    d = rng.integers(0, 1 << 32, 50000, dtype=np.uint64).astype(np.uint32)
    s[::7] = 0xFFFFFFFF
    d[::5] = 0xFFFFFFFF
    wins.append((s, d))
    big = (1 << 18) + 3
    wins.append((rng.integers(0, 1 << 20, big).astype(np.uint32), rng.integers(0, 1 << 20, big).astype(np.uint32)))
    # 8000 distinct links of a 8192-packet window (2 link partitions), all in partition 0
    cs = rng.integers(0, 1 << 32, 40000, dtype=np.uint64)
    cd = rng.integers(0, 1 << 32, 40000, dtype=np.uint64)
    keys = (cs << np.uint64(32)) | cd
    part = ((_fmix64(keys) >> np.uint64(40)) * np.uint64(2)) >> np.uint64(24)
    sel = np.unique(keys[part == 0])[:8000]
    sel = np.concatenate([sel, sel[:192]])
    rng.shuffle(sel)
    wins.append(((sel >> np.uint64(32)).astype(np.uint32), (sel & np.uint64(0xFFFFFFFF)).astype(np.uint32)))
    # 14000 distinct links with distinct sources (2 source partitions), all in source partition 0
    cand = rng.integers(0, 1 << 32, 60000, dtype=np.uint64).astype(np.uint32)
    sp = ((_fmix32(cand) >> np.uint64(14)) * np.uint64(2)) >> np.uint64(18)
    srcs = np.unique(cand[sp == 0])[:14000]
    wins.append((rng.permutation(srcs), rng.integers(0, 1 << 32, len(srcs), dtype=np.uint64).astype(np.uint32)))
    offsets = np.zeros(len(wins) + 1, np.uint64)
    offsets[1:] = np.cumsum([len(x) for x, _ in wins])
    w = sy.Windows(np.concatenate([x for x, _ in wins]), np.concatenate([y for _, y in wins]), offsets)
    c = ans.Context(0)
    try:
        c.set_tuning(agg_path=2, sum_path=2)
        flags = ans.BATCH_SUM if with_sum else 0
        for _ in range(2):  # twice: the second call replays the graph over the same scratch
            _, summ, quants = run_batch(ans, c, w, flags)
            exp = [oracle.window_quantities(*w.window(i)) for i in range(w.nwin)]
            for i in range(w.nwin):
                assert quants[i] == exp[i], f"window {i}"
            if with_sum:
                exp_sum = oracle.traffic_matrix(w.src, w.dst)
                assert_dcsr_equal(summ.to_numpy(), exp_sum, "sum")
                assert summ.quantities() == oracle.network_quantities(exp_sum)
                summ.free()
        # with per-window matrices the path does not apply: the sort runs
        check_batch(ans, c, synth.generate(5, nwin=5), check_sum=True)
    finally:
        c.close()
