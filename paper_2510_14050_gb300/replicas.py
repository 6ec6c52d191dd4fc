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
# mod the number of ranks, so every rank sends each link to the owner of its
# row (one all-to-all of (src << 32 | dst, count) pairs), and each owner adds
# the sorted pieces it receives.  Rows never straddle owners, so the owners'
# matrices together are exactly the global sum, row-partitioned.

import numpy as _np

_GOLDEN = 0x9E3779B1


def row_owner(row_ids, world: int):
    """Owner rank of each row (source address): a multiplicative hash of the
    address, so that consecutive or clustered sources spread over ranks."""
    h = (_np.asarray(row_ids, dtype=_np.uint64) * _GOLDEN) & 0xFFFFFFFF
    return ((h * world) >> 32).astype(_np.int64)


def partition_links(row_ids, row_ptr, col_ids, vals, world: int):
    """Split a DCSR matrix's links by the owner of their row: a list over
    ranks of (keys, values) with keys src << 32 | dst, each in DCSR order."""
    row_ids = _np.asarray(row_ids, dtype=_np.uint64)
    row_ptr = _np.asarray(row_ptr, dtype=_np.int64)
    counts = _np.diff(row_ptr)
    src = _np.repeat(row_ids, counts)
    keys = (src << _np.uint64(32)) | _np.asarray(col_ids, dtype=_np.uint64)
    own = _np.repeat(row_owner(row_ids, world), counts)
    vals = _np.asarray(vals, dtype=_np.uint64)
    return [(keys[own == r], vals[own == r]) for r in range(world)]


def exchange_links(parts, dist, device: str = "cpu"):
    """All-to-all of the link pieces: parts[r] goes to rank r; returns the
    pieces this rank received, one per sender, in rank order.  The buffers
    live on `device` ("cpu" for gloo, the rank's GPU for NCCL)."""
    import torch
    world = dist.get_world_size()
    send_n = torch.tensor([len(k) for k, _ in parts], dtype=torch.int64, device=device)
    recv_n = torch.empty(world, dtype=torch.int64, device=device)
    dist.all_to_all_single(recv_n, send_n)
    send_k = torch.from_numpy(_np.concatenate([k for k, _ in parts]).view(_np.int64)).to(device)
    send_v = torch.from_numpy(_np.concatenate([v for _, v in parts]).view(_np.int64)).to(device)
    sizes_out, sizes_in = send_n.tolist(), recv_n.tolist()
    total = int(sum(sizes_in))
    recv_k = torch.empty(total, dtype=torch.int64, device=device)
    recv_v = torch.empty(total, dtype=torch.int64, device=device)
    dist.all_to_all_single(recv_k, send_k, output_split_sizes=sizes_in, input_split_sizes=sizes_out)
    dist.all_to_all_single(recv_v, send_v, output_split_sizes=sizes_in, input_split_sizes=sizes_out)
    keys = recv_k.cpu().numpy().view(_np.uint64)
    vals = recv_v.cpu().numpy().view(_np.uint64)
    out, o = [], 0
    for n in sizes_in:
        out.append((keys[o:o + n], vals[o:o + n]))
        o += n
    return out


def keys_to_dcsr(keys, vals):
    """DCSR arrays of sorted, distinct link keys with their counts."""
    keys = _np.asarray(keys, dtype=_np.uint64)
    src = (keys >> _np.uint64(32)).astype(_np.uint32)
    col = (keys & _np.uint64(0xFFFFFFFF)).astype(_np.uint32)
    if len(keys) == 0:
        return _np.zeros(0, _np.uint32), _np.zeros(1, _np.uint64), col, _np.asarray(vals, _np.uint64)
    starts = _np.concatenate([[0], _np.nonzero(src[1:] != src[:-1])[0] + 1])
    row_ptr = _np.concatenate([starts, [len(keys)]]).astype(_np.uint64)
    return src[starts], row_ptr, col, _np.asarray(vals, _np.uint64)


def exchange_time_sum(ctx, partial, dist, device: str = "cpu"):
    """This rank's partition of the time sum over every rank's windows, from
    its own partial sum `partial` (an ans.Matrix): the links go to their
    rows' owners, and the pieces received are imported and added on this
    rank's device.  Returns an ans.Matrix holding the rows this rank owns.
    `device`: where the exchange buffers live (see exchange_links)."""
    world = dist.get_world_size()
    pieces = exchange_links(partition_links(*partial.to_numpy(), world), dist, device)
    mats = [ctx.import_matrix(*keys_to_dcsr(k, v)) for k, v in pieces]
    try:
        return ctx.sum_windows(mats)
    finally:
        for m in mats:
            m.free()
