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
