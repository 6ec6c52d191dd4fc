"""Host-side logic of the multi-GPU run: independent replicas.

Windows are independent (per-window DCSR and quantities need no data from
other windows), so N ranks each process their own batch of distinct windows
with no data-path collective.  The only cross-rank operations are timing: a
barrier on both sides of the timed region and the maximum elapsed time over
ranks; the whole-job rate is every rank's units over that maximum (weak
scaling: the per-rank work is fixed as N grows).
"""
from __future__ import annotations


def first_window(rank: int, nwin: int) -> int:
    """Index of rank's first window: rank r serves windows [r * nwin, (r+1) * nwin)
    of the seeded stream, so no two ranks see the same window."""
    return rank * nwin


def max_over_ranks(x: float, dist=None, device: str = "cpu") -> float:
    """Largest x over all ranks of the default process group (x itself when
    dist is None)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, dist=None, device: str = "cpu") -> float:
    """Sum of x over all ranks of the default process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units_all_ranks: float, elapsed_max_s: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's elapsed time."""
    return units_all_ranks / elapsed_max_s


# ---- the time sum across ranks: one exchange step ---------------------------
#
# Each rank holds the time sum of its own windows.  The global sum is owned
# in row (source) partitions: a row's owner is a hash of its source address
# mod the number of ranks, so every rank sends each of its rows to the owner
# (the library splits the partial sum by owner; one all-to-all of the DCSR
# pieces), and each owner adds the pieces it receives.  Rows never straddle owners, so the owners'
# matrices together are exactly the global sum, row-partitioned.

import numpy as _np

_GOLDEN = 0x9E3779B1


def row_owner(row_ids, world: int):
    """Owner rank of each row (source address): a multiplicative hash of the
    address, so that consecutive or clustered sources spread over ranks."""
    h = (_np.asarray(row_ids, dtype=_np.uint64) * _GOLDEN) & 0xFFFFFFFF
    return ((h * world) >> 32).astype(_np.int64)


def exchange_pieces(pieces, dist, device: str = "cpu"):
    """All-to-all of DCSR pieces: pieces[r] = (row_ids, row_ptr, col_ids,
    vals) numpy arrays for rank r; returns the pieces this rank received, one
    per sender, in rank order.  The buffers live on `device` ("cpu" for
    gloo, the rank's GPU for NCCL)."""
    import torch
    world = dist.get_world_size()
    out = [[None] * 4 for _ in range(world)]
    for a in range(4):
        send = [_np.ascontiguousarray(p[a]) for p in pieces]
        item = send[0].dtype
        as_i = _np.int32 if item.itemsize == 4 else _np.int64
        send_n = torch.tensor([len(x) for x in send], dtype=torch.int64, device=device)
        recv_n = torch.empty(world, dtype=torch.int64, device=device)
        dist.all_to_all_single(recv_n, send_n)
        sizes_out, sizes_in = send_n.tolist(), recv_n.tolist()
        buf = torch.from_numpy(_np.concatenate(send).view(as_i)).to(device)
        recv = torch.empty(int(sum(sizes_in)), dtype=buf.dtype, device=device)
        dist.all_to_all_single(recv, buf, output_split_sizes=sizes_in, input_split_sizes=sizes_out)
        got = recv.cpu().numpy().view(item)
        o = 0
        for r, n in enumerate(sizes_in):
            out[r][a] = got[o:o + n]
            o += n
    return [tuple(x) for x in out]


def exchange_time_sum(ctx, partial, dist, device: str = "cpu"):
    """This rank's partition of the time sum over every rank's windows, from
    its own partial sum `partial` (an ans.Matrix): the library splits the
    partial sum's rows by owner (ans_matrix_split_rows), each piece goes to
    its owner (host-staged all-to-all of the DCSR arrays), and the pieces
    received are imported and added on this rank's device.  Returns an
    ans.Matrix holding exactly the rows this rank owns."""
    world = dist.get_world_size()
    parts = ctx.split_rows(partial, world)
    try:
        pieces = [p.to_numpy() for p in parts]
    finally:
        for p in parts:
            p.free()
    received = exchange_pieces(pieces, dist, device)
    mats = [ctx.import_matrix(*piece) for piece in received]
    try:
        return ctx.sum_windows(mats)
    finally:
        for m in mats:
            m.free()
