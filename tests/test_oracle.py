"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself:
  * hand-worked windows (tests/golden/, from the definitions of Table I and
    Sec. IV-B/IV-C);
  * O(P^2) brute force written with plain Python loops over the packets;
  * closed forms (all-identical, all-distinct, stars) and invariants
    (conservation, bounds, transpose symmetry, permutation invariance,
    additivity of the time sum);
  * planted mistakes: mutated copies of the oracle must fail the pins.
"""
import numpy as np
import pytest

import oracle
from oracle import ans_oracle
from oracle import QUANTITY_NAMES
from tests import golden_io

# ------------------------------------------------------------ brute force --


def brute_quantities(src, dst):
    """The nine quantities by scanning the packet list, O(P^2), no sorting."""
    s = [int(v) for v in src]
    d = [int(v) for v in dst]
    p = len(s)
    first_link = [all((s[j], d[j]) != (s[k], d[k]) for j in range(k)) for k in range(p)]
    first_src = [all(s[j] != s[k] for j in range(k)) for k in range(p)]
    first_dst = [all(d[j] != d[k] for j in range(k)) for k in range(p)]
    link_pk = [sum(1 for j in range(p) if (s[j], d[j]) == (s[k], d[k])) for k in range(p)]
    src_pk = [sum(1 for j in range(p) if s[j] == s[k]) for k in range(p)]
    dst_pk = [sum(1 for j in range(p) if d[j] == d[k]) for k in range(p)]
    fan_out = [sum(1 for j in range(p) if s[j] == s[k] and first_link[j]) for k in range(p)]
    fan_in = [sum(1 for j in range(p) if d[j] == d[k] and first_link[j]) for k in range(p)]
    return {
        "valid_packets": p,
        "unique_links": sum(first_link),
        "max_link_packets": max(link_pk, default=0),
        "unique_sources": sum(first_src),
        "max_source_packets": max(src_pk, default=0),
        "max_source_fanout": max(fan_out, default=0),
        "unique_destinations": sum(first_dst),
        "max_destination_packets": max(dst_pk, default=0),
        "max_destination_fanin": max(fan_in, default=0),
    }


def brute_dcsr(src, dst):
    """DCSR by scanning: distinct links in (src, dst) order, counts by scanning."""
    pairs = [(int(a), int(b)) for a, b in zip(src, dst)]
    links = []
    for pr in pairs:
        if pr not in links:
            links.append(pr)
    links.sort()
    row_ids, row_ptr = [], []
    for i, (a, _) in enumerate(links):
        if not row_ids or row_ids[-1] != a:
            row_ids.append(a)
            row_ptr.append(i)
    row_ptr.append(len(links))
    col_ids = [b for _, b in links]
    vals = [sum(1 for pr in pairs if pr == lk) for lk in links]
    return row_ids, row_ptr, col_ids, vals


def as_lists(m):
    return ([int(v) for v in m.row_ids], [int(v) for v in m.row_ptr],
            [int(v) for v in m.col_ids], [int(v) for v in m.vals])


def check_dcsr_canonical(m):
    assert m.row_ids.dtype == np.uint32 and m.col_ids.dtype == np.uint32
    assert m.row_ptr.dtype == np.uint64 and m.vals.dtype == np.uint64
    assert len(m.row_ptr) == m.nrows + 1 and int(m.row_ptr[0]) == 0 and int(m.row_ptr[-1]) == m.nnz
    assert np.all(np.diff(m.row_ids.astype(np.int64)) > 0)
    assert np.all(np.diff(m.row_ptr.astype(np.int64)) > 0)
    for r in range(m.nrows):
        a, b = int(m.row_ptr[r]), int(m.row_ptr[r + 1])
        assert np.all(np.diff(m.col_ids[a:b].astype(np.int64)) > 0)
    assert np.all(m.vals > 0)


# ------------------------------------------------------------ golden files --


@pytest.mark.parametrize("name", golden_io.FIXTURES)
def test_golden_window(name):
    (win,), exp = golden_io.load(name)
    m = oracle.traffic_matrix(*win)
    check_dcsr_canonical(m)
    assert as_lists(m) == (exp["row_ids"], exp["row_ptr"], exp["col_ids"], exp["vals"])
    q = oracle.network_quantities(m)
    assert q == {k: exp[k][0] for k in QUANTITY_NAMES}


def test_golden_time_sum():
    wins, exp = golden_io.load("time_sum.txt")
    mats = [oracle.traffic_matrix(*w) for w in wins]
    s = oracle.sum_matrices(mats)
    check_dcsr_canonical(s)
    assert as_lists(s) == (exp["sum_row_ids"], exp["sum_row_ptr"], exp["sum_col_ids"], exp["sum_vals"])
    assert oracle.network_quantities(s) == {k: exp["sum_" + k][0] for k in QUANTITY_NAMES}


# ------------------------------------------------------------ brute force --


def _random_window(rng, p, pool_s, pool_d, extremes):
    cand_s = rng.integers(0, 2**32, size=pool_s, dtype=np.uint64).astype(np.uint32)
    cand_d = rng.integers(0, 2**32, size=pool_d, dtype=np.uint64).astype(np.uint32)
    if extremes:
        cand_s[0], cand_d[-1] = 0, 0xFFFFFFFF
        if pool_s > 1:
            cand_s[1] = 0xFFFFFFFF
        if pool_d > 1:
            cand_d[0] = 0
    src = cand_s[rng.integers(0, pool_s, size=p)]
    dst = cand_d[rng.integers(0, pool_d, size=p)]
    return src, dst


@pytest.mark.parametrize("seed", range(40))
def test_brute_force_random(seed):
    rng = np.random.default_rng(seed)
    p = int(rng.integers(0, 257))
    pool_s = int(rng.integers(1, 24))
    pool_d = int(rng.integers(1, 24))
    src, dst = _random_window(rng, p, pool_s, pool_d, extremes=seed % 3 == 0)
    m = oracle.traffic_matrix(src, dst)
    check_dcsr_canonical(m)
    assert as_lists(m) == tuple(brute_dcsr(src, dst))
    assert oracle.network_quantities(m) == brute_quantities(src, dst)


@pytest.mark.parametrize("seed", range(6))
def test_brute_force_time_sum(seed):
    rng = np.random.default_rng(100 + seed)
    wins = [_random_window(rng, int(rng.integers(0, 80)), 6, 9, extremes=True) for _ in range(4)]
    s = oracle.sum_matrices([oracle.traffic_matrix(*w) for w in wins])
    cat_s = np.concatenate([w[0] for w in wins])
    cat_d = np.concatenate([w[1] for w in wins])
    assert as_lists(s) == tuple(brute_dcsr(cat_s, cat_d))
    assert oracle.network_quantities(s) == brute_quantities(cat_s, cat_d)


# ------------------------------------------------------------ closed forms --


def test_empty_window():
    m = oracle.traffic_matrix(np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    assert m.nrows == 0 and m.nnz == 0 and list(m.row_ptr) == [0]
    assert oracle.network_quantities(m) == dict.fromkeys(QUANTITY_NAMES, 0)
    assert oracle.sum_matrices([m, m]).nnz == 0


def test_single_packet():
    q = oracle.window_quantities(np.array([5], np.uint32), np.array([5], np.uint32))
    assert q == dict.fromkeys(QUANTITY_NAMES, 1)


def test_all_identical():
    p = 1000
    q = oracle.window_quantities(np.full(p, 7, np.uint32), np.full(p, 0xFFFFFFFF, np.uint32))
    assert q == {"valid_packets": p, "unique_links": 1, "max_link_packets": p, "unique_sources": 1,
                 "max_source_packets": p, "max_source_fanout": 1, "unique_destinations": 1,
                 "max_destination_packets": p, "max_destination_fanin": 1}


def test_all_distinct_permutation():
    rng = np.random.default_rng(3)
    p = 5000
    src = rng.permutation(p).astype(np.uint32) * np.uint32(977)
    dst = rng.permutation(p).astype(np.uint32) + np.uint32(123456)
    q = oracle.window_quantities(src, dst)
    assert q == {"valid_packets": p, "unique_links": p, "max_link_packets": 1, "unique_sources": p,
                 "max_source_packets": 1, "max_source_fanout": 1, "unique_destinations": p,
                 "max_destination_packets": 1, "max_destination_fanin": 1}


def test_star_and_reverse_star():
    k = 3000
    src = np.full(k, 42, np.uint32)
    dst = np.arange(k, dtype=np.uint32) * np.uint32(65537)
    q = oracle.window_quantities(src, dst)
    assert (q["unique_sources"], q["max_source_fanout"], q["max_source_packets"]) == (1, k, k)
    assert (q["unique_destinations"], q["max_destination_fanin"], q["max_destination_packets"]) == (k, 1, 1)
    qt = oracle.window_quantities(dst, src)
    assert (qt["unique_destinations"], qt["max_destination_fanin"], qt["max_destination_packets"]) == (1, k, k)
    assert (qt["unique_sources"], qt["max_source_fanout"]) == (k, 1)


# ------------------------------------------------------------ invariants ---


def _synth_windows(cfg, nwin, sizes=None):
    synth = pytest.importorskip("paper_2510_14050_gb300.synth")
    return synth.generate(cfg, nwin=nwin, sizes=sizes)


def check_invariants(src, dst, m, q):
    vals = m.vals.astype(np.uint64)
    nv = q["valid_packets"]
    assert nv == len(src)
    assert int(vals.sum()) == nv                              # sum of rows == N_V
    assert q["unique_links"] <= nv
    assert q["unique_sources"] <= q["unique_links"] and q["unique_destinations"] <= q["unique_links"]
    assert q["max_source_fanout"] <= q["unique_destinations"]
    assert q["max_destination_fanin"] <= q["unique_sources"]
    assert q["max_link_packets"] <= min(q["max_source_packets"], q["max_destination_packets"]) <= nv
    if nv:
        assert q["max_source_packets"] * q["unique_sources"] >= nv
        assert q["max_destination_packets"] * q["unique_destinations"] >= nv
    # column sums (via the transposed matrix) also add up to N_V
    mt = oracle.traffic_matrix(dst, src)
    assert int(mt.vals.sum()) == nv


@pytest.mark.parametrize("cfg,sizes", [(1, [4096]), (2, [3000, 5000]), (3, [1024, 20000]), (4, [4096]),
                                       (5, [4096, 7000])])
def test_invariants_and_symmetry(cfg, sizes):
    w = _synth_windows(cfg, len(sizes), sizes)
    mats = []
    for i in range(w.nwin):
        s, d = w.window(i)
        m = oracle.traffic_matrix(s, d)
        check_dcsr_canonical(m)
        q = oracle.network_quantities(m)
        check_invariants(s, d, m, q)
        # transpose symmetry: swapping src and dst swaps the row and column statistics
        qt = oracle.window_quantities(d, s)
        assert (qt["unique_sources"], qt["max_source_packets"], qt["max_source_fanout"]) == \
            (q["unique_destinations"], q["max_destination_packets"], q["max_destination_fanin"])
        assert (qt["unique_destinations"], qt["max_destination_packets"], qt["max_destination_fanin"]) == \
            (q["unique_sources"], q["max_source_packets"], q["max_source_fanout"])
        assert qt["unique_links"] == q["unique_links"] and qt["max_link_packets"] == q["max_link_packets"]
        # permutation invariance of packet order
        perm = np.random.default_rng(i).permutation(len(s))
        mp = oracle.traffic_matrix(s[perm], d[perm])
        assert all(np.array_equal(a, b) for a, b in zip(m, mp))
        mats.append(m)
    # additivity: sum of window matrices == matrix of the concatenated stream
    total = oracle.sum_matrices(mats)
    whole = oracle.traffic_matrix(w.src, w.dst)
    assert all(np.array_equal(a, b) for a, b in zip(total, whole))


def test_batch_helper_matches_per_window():
    w = _synth_windows(2, 3, [2000, 0, 3000])
    mats, quants, total = oracle.batch(w.src, w.dst, w.offsets)
    assert mats[1].nnz == 0 and quants[1] == dict.fromkeys(QUANTITY_NAMES, 0)
    arr = oracle.quantities_array(quants)
    assert arr.shape == (3, 9) and int(arr[0, 0]) == 2000 and int(arr[2, 0]) == 3000
    assert total.nnz == oracle.traffic_matrix(w.src, w.dst).nnz


def test_large_counts_stay_exact():
    # values above 2^53 must not pass through floating point
    big = np.uint64(2**60 + 12345)
    m = oracle.DCSR(np.array([1, 2], np.uint32), np.array([0, 2, 3], np.uint64),
                    np.array([5, 6, 5], np.uint32), np.array([big, 1, big], np.uint64))
    q = oracle.network_quantities(m)
    assert q["valid_packets"] == int(big) * 2 + 1
    assert q["max_source_packets"] == int(big) + 1
    assert q["max_destination_packets"] == int(big) * 2
    s = oracle.sum_matrices([m, m])
    assert [int(v) for v in s.vals] == [2 * int(big), 2, 2 * int(big)]


# ------------------------------------------------------------ planted mistakes


def _pins_pass(tm, nq, sm):
    """Run the golden + brute pins against a (possibly mutated) oracle."""
    try:
        for name in golden_io.FIXTURES:
            (win,), exp = golden_io.load(name)
            m = tm(*win)
            if as_lists(m) != (exp["row_ids"], exp["row_ptr"], exp["col_ids"], exp["vals"]):
                return False
            if nq(m) != {k: exp[k][0] for k in QUANTITY_NAMES}:
                return False
        wins, exp = golden_io.load("time_sum.txt")
        s = sm([tm(*w) for w in wins])
        if as_lists(s) != (exp["sum_row_ids"], exp["sum_row_ptr"], exp["sum_col_ids"], exp["sum_vals"]):
            return False
        rng = np.random.default_rng(7)
        for _ in range(5):
            src, dst = _random_window(rng, 60, 5, 7, extremes=True)
            if nq(tm(src, dst)) != brute_quantities(src, dst):
                return False
    except Exception:
        return False
    return True


def test_pins_accept_the_oracle():
    assert _pins_pass(oracle.traffic_matrix, oracle.network_quantities, oracle.sum_matrices)


def _mut_transposed(src, dst):
    return ans_oracle.traffic_matrix(dst, src)


def _mut_no_counts(src, dst):
    m = ans_oracle.traffic_matrix(src, dst)
    return m._replace(vals=np.ones_like(m.vals))


def _mut_row_ptr_shift(src, dst):
    m = ans_oracle.traffic_matrix(src, dst)
    rp = m.row_ptr.copy()
    rp[1:-1] += 1
    return m._replace(row_ptr=rp)


def _nq_fanout_as_rowsum(m):
    q = ans_oracle.network_quantities(m)
    q["max_source_fanout"] = q["max_source_packets"]
    return q


def _nq_fanin_as_distinct_rows(m):
    q = ans_oracle.network_quantities(m)
    q["max_destination_fanin"] = min(q["max_destination_fanin"], 1)  # Table I's literal zero-norm reading
    return q


def _nq_unique_dst_from_rows(m):
    q = ans_oracle.network_quantities(m)
    q["unique_destinations"] = q["unique_sources"]
    return q


def _sm_keep_max(mats):
    # a time sum that takes the max over windows instead of adding counts
    s = ans_oracle.sum_matrices(mats)
    return s._replace(vals=np.minimum(s.vals, np.uint64(2)))


@pytest.mark.parametrize("tm,nq,sm", [
    (_mut_transposed, oracle.network_quantities, oracle.sum_matrices),
    (_mut_no_counts, oracle.network_quantities, oracle.sum_matrices),
    (_mut_row_ptr_shift, oracle.network_quantities, oracle.sum_matrices),
    (oracle.traffic_matrix, _nq_fanout_as_rowsum, oracle.sum_matrices),
    (oracle.traffic_matrix, _nq_fanin_as_distinct_rows, oracle.sum_matrices),
    (oracle.traffic_matrix, _nq_unique_dst_from_rows, oracle.sum_matrices),
    (oracle.traffic_matrix, oracle.network_quantities, _sm_keep_max),
])
def test_pins_reject_planted_mistakes(tm, nq, sm):
    assert not _pins_pass(tm, nq, sm)
