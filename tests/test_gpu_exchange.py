"""The exchange step of a time sum computed on several devices (Sec. III-A,
Fig. 4), on the GPU: the library's row split of a matrix by owner rank
equals the oracle's row partition, and two processes -- two ranks of a gloo
group sharing this one GPU, each running only its own independent kernels --
each build their windows' time sum with libans, exchange the pieces
host-staged, and end with exactly the rows they own of the global sum."""
import os
import socket

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _owner(rows, world):
    h = (np.asarray(rows, dtype=np.uint64) * np.uint64(0x9E3779B1)) & np.uint64(0xFFFFFFFF)
    return ((h * np.uint64(world)) >> np.uint64(32)).astype(np.int64)


def _owned_rows(m, world, r):
    own = _owner(m.row_ids, world) == r
    counts = np.diff(m.row_ptr.astype(np.int64))
    keep = np.repeat(own, counts)
    rp = np.concatenate([[0], np.cumsum(counts[own])]).astype(np.uint64)
    return oracle.DCSR(m.row_ids[own], rp, m.col_ids[keep], m.vals[keep])


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


@pytest.mark.parametrize("nparts", [1, 3, 8, 64])
def test_row_split_equals_the_oracle_partition(nparts):
    from paper_2510_14050_gb300 import ans, synth
    w = synth.generate(2, nwin=8)
    ctx = ans.Context(0)
    try:
        _, summ, tk = ctx.batch_submit(_dev(w.src), _dev(w.dst), w.offsets, ans.BATCH_SUM)
        ctx.wait(tk)
        exp = oracle.traffic_matrix(w.src, w.dst)
        parts = ctx.split_rows(summ, nparts)
        for r, p in enumerate(parts):
            want = _owned_rows(exp, nparts, r)
            for name, a, b in zip(want._fields, p.to_numpy(), want):
                assert np.array_equal(a, b), f"part {r}: {name}"
            assert p.quantities() == oracle.network_quantities(want)
            p.free()
        summ.free()
        # an empty matrix splits into empty pieces
        _, e, tk = ctx.batch_submit(_dev([0]), _dev([0]), np.zeros(1, np.uint64), ans.BATCH_SUM)
        ctx.wait(tk)
        for p in ctx.split_rows(e, nparts):
            assert p.view()[:2] == (0, 0)
            p.free()
        e.free()
    finally:
        ctx.close()


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2510_14050_gb300 import ans, replicas, synth
        torch.cuda.set_device(0)
        w = synth.generate(2, nwin=4, first_window=replicas.first_window(rank, 4))
        ctx = ans.Context(0)
        try:
            _, partial, tk = ctx.batch_submit(_dev(w.src), _dev(w.dst), w.offsets, ans.BATCH_SUM)
            ctx.wait(tk)
            owned = replicas.exchange_time_sum(ctx, partial, dist)
            out[rank] = tuple(a.tolist() for a in owned.to_numpy())
            out[f"q{rank}"] = owned.quantities()
            owned.free()
            partial.free()
        finally:
            ctx.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_ranks_exchange_their_time_sums_on_the_gpu(world):
    import torch.multiprocessing as mp
    from paper_2510_14050_gb300 import replicas, synth
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    with mp.get_context("spawn").Manager() as mgr:  # no fork after CUDA is initialised
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    srcs, dsts = [], []
    for r in range(world):
        w = synth.generate(2, nwin=4, first_window=replicas.first_window(r, 4))
        srcs.append(w.src)
        dsts.append(w.dst)
    exp = oracle.traffic_matrix(np.concatenate(srcs), np.concatenate(dsts))
    for r in range(world):
        want = _owned_rows(exp, world, r)
        for name, a, b in zip(want._fields, res[r], want):
            assert np.array_equal(np.asarray(a, dtype=b.dtype), b), f"rank {r}: {name}"
        assert res[f"q{r}"] == oracle.network_quantities(want)
