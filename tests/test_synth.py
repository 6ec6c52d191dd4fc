"""The seeded generator (no GPU): determinism and the workload recipe."""
import numpy as np
import pytest

from paper_2510_14050_gb300 import synth


def test_deterministic_and_thread_independent():
    a = synth.generate(2, nwin=3, threads=1)
    b = synth.generate(2, nwin=3, threads=8)
    assert np.array_equal(a.src, b.src) and np.array_equal(a.dst, b.dst)
    c = synth.generate(2, nwin=3, seed=1)
    assert not np.array_equal(a.src, c.src)
    # window w does not depend on which other windows are generated with it
    d = synth.generate(2, nwin=1, first_window=2)
    s, t = a.window(2)
    assert np.array_equal(d.src, s) and np.array_equal(d.dst, t)


@pytest.mark.parametrize("s,n", [(1.2, 1 << 16), (1.05, 1 << 32), (1.3, 1 << 22), (0.7, 50)])
def test_zipf_head_frequencies(s, n):
    count = 1 << 20
    r = synth.zipf_ranks(s, n, count)
    assert r.min() >= 1 and r.max() <= n
    if n <= 1 << 22:
        h = np.sum(np.arange(1, n + 1, dtype=np.float64) ** -s)
    else:  # Euler-Maclaurin tail for the generalised harmonic number
        k = np.arange(1, 100001, dtype=np.float64)
        m = 100000.0
        h = np.sum(k ** -s) + ((n ** (1 - s)) - m ** (1 - s)) / (1 - s) - 0.5 * m ** -s + 0.5 * n ** -s
    for k in (1, 2, 3, 10):
        p = k ** -s / h
        sd = np.sqrt(p * (1 - p) / count)
        assert abs(np.mean(r == k) - p) < 5 * sd + 1e-9


def test_config_sizes():
    assert list(synth.window_sizes(1, 1)) == [1 << 17]
    assert set(synth.window_sizes(2, 64)) == {1 << 17}
    s3 = synth.window_sizes(3, 1024)
    assert s3.min() >= 1 << 10 and s3.max() <= 1 << 20
    assert 1.2e8 < s3.sum() < 1.9e8          # E[P] = (2^20 - 2^10) / (10 ln 2)
    s5 = synth.window_sizes(5, 5000)
    assert s5.min() >= 1 << 12 and s5.max() <= 1 << 17


def test_addresses_are_rank_images():
    w = synth.generate(1)
    k = synth.rank_to_addr(np.arange(1, (1 << 16) + 1))
    assert len(np.unique(k)) == 1 << 16
    assert np.isin(w.src, k).all() and np.isin(w.dst, k).all()


def test_cfg2_bursts():
    p = 1 << 17
    w = synth.generate(2, nwin=1)
    s, d = w.window(0)
    assert len(s) == p
    # runs of identical consecutive pairs of length >= 2 cover at least floor(0.05 P) packets
    same = (s[1:] == s[:-1]) & (d[1:] == d[:-1])
    assert same.sum() >= int(0.05 * p) - int(0.05 * p) // 2


def test_cfg3_heavy_hitter_and_scanners():
    sizes = [1 << 15]
    w = synth.generate(3, nwin=1, sizes=sizes)
    s, d = w.window(0)
    hh = np.uint32(0xC0A80001)
    assert (s == hh).sum() >= int(0.10 * sizes[0])
    # one scanner (P / 2^14 = 2) with consecutive destinations exists: some source hits
    # at least 16 distinct consecutive addresses
    pool = synth.rank_to_addr(np.arange((1 << 24) + 1, (1 << 24) + 1 + 16777))
    scan = np.isin(s, pool)
    assert scan.sum() >= 16
    assert scan.sum() <= int(0.10 * sizes[0]) + 64


def test_arrivals_poisson():
    t = synth.arrivals(1000.0, 20000)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 1e-3) < 5e-5
