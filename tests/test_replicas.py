"""The multi-GPU run is replicas: ranks take disjoint windows, share nothing
on the data path, and agree on the slowest rank's time.  Two gloo ranks on
the CPU exercise that host-side logic (no GPU)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2510_14050_gb300 import replicas, synth
        nwin = 3
        w = synth.generate(5, nwin=nwin, first_window=replicas.first_window(rank, nwin))
        keys = np.unique((w.src.astype(np.uint64) << 32) | w.dst)
        elapsed = 0.5 + rank  # rank 1 is the slow one
        dist.barrier()
        t = replicas.max_over_ranks(elapsed, dist)
        units = replicas.sum_over_ranks(float(w.total), dist)
        out[rank] = (t, replicas.job_rate(units, t), int(w.total), keys[:64].tolist(),
                     replicas.first_window(rank, nwin), units)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_disjoint_windows_and_agree_on_time():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:  # no fork after CUDA is initialised
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    both = res[0][2] + res[1][2]
    for r in range(world):
        t, rate, total, _, first, units = res[r]
        assert t == pytest.approx(1.5)  # both ranks see the slowest rank's time
        assert first == 3 * r
        assert units == both
        # the whole-job rate counts every rank's packets over the slowest time
        assert rate == pytest.approx(both / 1.5)
    # different windows on each rank (seeded by window index)
    assert res[0][3] != res[1][3]


def test_single_process_helpers():
    from paper_2510_14050_gb300 import replicas
    assert replicas.max_over_ranks(2.5) == 2.5
    assert replicas.job_rate(400.0, 2.0) == 200.0
    assert replicas.sum_over_ranks(3.0) == 3.0
    assert replicas.first_window(0, 64) == 0 and replicas.first_window(3, 64) == 192


def _owned_rows(m, world, r):
    """Rows of DCSR m whose owner is rank r (the test's own row split)."""
    import oracle
    from paper_2510_14050_gb300 import replicas
    own = replicas.row_owner(m.row_ids, world) == r
    counts = np.diff(m.row_ptr.astype(np.int64))
    keep = np.repeat(own, counts)
    rp = np.concatenate([[0], np.cumsum(counts[own])]).astype(np.uint64)
    return oracle.DCSR(m.row_ids[own], rp, m.col_ids[keep], m.vals[keep])


def _exchange_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2510_14050_gb300 import replicas, synth
        w = synth.generate(5, nwin=3, first_window=replicas.first_window(rank, 3))
        partial = oracle.sum_matrices([oracle.traffic_matrix(*w.window(i)) for i in range(w.nwin)])
        pieces = [tuple(_owned_rows(partial, world, r)) for r in range(world)]
        received = replicas.exchange_pieces(pieces, dist)
        owned = oracle.sum_matrices([oracle.DCSR(*p) for p in received])
        out[rank] = tuple(a.tolist() for a in owned)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_exchange_their_time_sums(world):
    """The one exchange step of a multi-rank time sum: rows go to their
    owners as DCSR pieces; the owners' matrices are the row partition of the
    global sum (checked against the oracle's sum of every rank's windows)."""
    import oracle
    from paper_2510_14050_gb300 import replicas, synth
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:  # no fork after CUDA is initialised
        out = mgr.dict()
        mp.spawn(_exchange_main, args=(world, port, out), nprocs=world, join=True)
        res = {r: tuple(np.asarray(a) for a in out[r]) for r in range(world)}
    mats = []
    for r in range(world):
        w = synth.generate(5, nwin=3, first_window=replicas.first_window(r, 3))
        mats += [oracle.traffic_matrix(*w.window(i)) for i in range(w.nwin)]
    exp = oracle.sum_matrices(mats)
    for r in range(world):
        want = _owned_rows(exp, world, r)
        for a, b in zip(res[r], want):
            assert np.array_equal(np.asarray(a, dtype=np.uint64), np.asarray(b, dtype=np.uint64))
    assert sum(len(res[r][0]) for r in range(world)) == exp.nrows
