"""Host-side parts of the serving loop: the arrival schedule, the window
pool and the latency summary (no GPU)."""
import numpy as np
import pytest

from paper_2510_14050_gb300 import serve


def test_poisson_schedule_is_ordered_and_has_the_rate():
    rate, n, pool = 5000.0, 20000, 37
    t, order = serve.poisson_schedule(rate, n, pool, seed=3)
    assert t.shape == (n,) and order.shape == (n,)
    assert np.all(np.diff(t) >= 0) and t[0] >= 0
    gaps = np.diff(np.concatenate([[0.0], t]))
    # exponential inter-arrival times: mean 1/rate, standard deviation 1/rate
    assert abs(gaps.mean() * rate - 1.0) < 0.05
    assert abs(gaps.std() * rate - 1.0) < 0.05
    assert order.min() >= 0 and order.max() < pool
    assert len(set(order[:pool].tolist())) == pool  # the schedule walks the whole pool
    t2, _ = serve.poisson_schedule(rate, n, pool, seed=3)
    assert np.array_equal(t, t2)  # seeded
    with pytest.raises(ValueError):
        serve.poisson_schedule(0.0, 10, pool)


def test_pool_windows_have_serving_sizes():
    src = serve.pool_source(64, seed=1)
    sizes = np.diff(src.offsets.astype(np.int64))
    assert len(sizes) == 64 and src.offsets[0] == 0
    assert sizes.min() >= 1 << 12 and sizes.max() <= 1 << 17
    assert len(src.src) == len(src.dst) == int(src.offsets[-1])
    assert src.size(5) == sizes[5]


def test_latency_summary():
    lat = np.linspace(0.001, 0.1, 100)
    st = serve.ServeStats(latencies_s=lat, quantities=np.zeros((100, 9), np.uint64), packets=10 ** 6, wall_s=2.0,
                          batches=7, admission_stalls=1, max_queue=4)
    s = st.summary()
    assert s["windows"] == 100 and s["batches"] == 7 and s["admission_stalls"] == 1 and s["max_queue"] == 4
    assert s["p50_ms"] == pytest.approx(np.percentile(lat, 50) * 1e3, abs=1e-3)
    assert s["p99_ms"] == pytest.approx(np.percentile(lat, 99) * 1e3, abs=1e-3)
    assert s["max_ms"] == pytest.approx(100.0)
    assert s["sustained_packets_per_s"] == pytest.approx(5e5)
    empty = serve.ServeStats(latencies_s=np.zeros(0), quantities=np.zeros((0, 9), np.uint64), packets=0,
                             wall_s=0.0, batches=0, admission_stalls=0, max_queue=0).summary()
    assert empty["windows"] == 0 and empty["p99_ms"] == 0.0 and empty["sustained_packets_per_s"] == 0.0
