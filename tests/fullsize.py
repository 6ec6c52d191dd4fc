"""Oracle checks of full-size batches, spread over the host's cores.

The time sum of a batch (Table I: A_t summed over t) is checked slice by
slice: rows [lo, hi) of sum_t A_t are exactly the traffic matrix of the
packets whose source lies in [lo, hi) (each row only counts its own
packets), so the oracle's ``traffic_matrix`` of those packets must equal the
GPU sum's rows in that range, array by array.  Slices that partition the
2^32 source space cover the whole sum.  Likewise the column quantities of the
sum restricted to destinations in [lo, hi) are those of the oracle's matrix
of the packets whose destination lies there.  Slices run on a thread pool:
numpy releases the interpreter lock in its masks and sorts.

Only the oracle computes expected values here; the GPU arrays are only
compared against them.
"""
from __future__ import annotations

import concurrent.futures as cf
import os

import numpy as np

import oracle

SPACE = 1 << 32


def _threads():
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except Exception:
        return os.cpu_count() or 1


def _select(key, lo, hi):
    return (key >= lo) & (key < hi) if hi < SPACE else (key >= lo)


def rows_of(gpu, lo, hi):
    """Rows [lo, hi) of a DCSR given as (row_ids, row_ptr, col_ids, vals)
    numpy arrays, as a DCSR of their own."""
    r, p, c, v = gpu
    r0, r1 = np.searchsorted(r, lo), np.searchsorted(r, hi) if hi < SPACE else len(r)
    u0, u1 = int(p[r0]), int(p[r1])
    return oracle.DCSR(r[r0:r1], p[r0:r1 + 1] - np.uint64(u0), c[u0:u1], v[u0:u1])


def _check_rows(src, dst, gpus, lo, hi):
    m = _select(src, lo, hi)
    exp = oracle.traffic_matrix(src[m], dst[m])
    bad = []
    for k, g in enumerate(gpus):
        got = rows_of(g, lo, hi)
        for name, a, b in zip(exp._fields, got, exp):
            if not np.array_equal(a, b):
                bad.append((k, lo, hi, name))
                break
    return bad, oracle.network_quantities(exp)


def _check_cols(src, dst, lo, hi):
    m = _select(dst, lo, hi)
    return oracle.network_quantities(oracle.traffic_matrix(src[m], dst[m]))


def check_time_sum(src, dst, gpus, slices: int):
    """Compare every GPU time sum in `gpus` (each a (row_ids, row_ptr,
    col_ids, vals) tuple) with the oracle's sum of the packets (src, dst),
    over `slices` equal source slices; also build the sum's nine quantities
    from the oracle's row slices and destination slices.  Returns (list of
    mismatches, expected quantities of the sum)."""
    edges = [SPACE * i // slices for i in range(slices + 1)]
    for g in gpus:  # the row slices partition the stored rows only if the DCSR frames agree
        r, p, c, v = g
        assert p[0] == 0 and int(p[-1]) == len(c) == len(v) and len(p) == len(r) + 1
    with cf.ThreadPoolExecutor(_threads()) as ex:
        rows = list(ex.map(lambda i: _check_rows(src, dst, gpus, edges[i], edges[i + 1]), range(slices)))
        cols = list(ex.map(lambda i: _check_cols(src, dst, edges[i], edges[i + 1]), range(slices)))
    bad = [b for r in rows for b in r[0]]
    rq = [r[1] for r in rows]
    q = {
        "valid_packets": sum(x["valid_packets"] for x in rq),
        "unique_links": sum(x["unique_links"] for x in rq),
        "max_link_packets": max(x["max_link_packets"] for x in rq),
        "unique_sources": sum(x["unique_sources"] for x in rq),
        "max_source_packets": max(x["max_source_packets"] for x in rq),
        "max_source_fanout": max(x["max_source_fanout"] for x in rq),
        "unique_destinations": sum(x["unique_destinations"] for x in cols),
        "max_destination_packets": max(x["max_destination_packets"] for x in cols),
        "max_destination_fanin": max(x["max_destination_fanin"] for x in cols),
    }
    return bad, q


def window_quantities(w):
    """The oracle's quantities of every window of `w`, on all cores."""
    def one(i):
        return oracle.window_quantities(*w.window(i))
    with cf.ThreadPoolExecutor(_threads()) as ex:
        return list(ex.map(one, range(w.nwin), chunksize=16))


def window_matrices(w, ids):
    """The oracle's DCSR of windows `ids` of `w`, on all cores."""
    def one(i):
        return oracle.traffic_matrix(*w.window(i))
    with cf.ThreadPoolExecutor(_threads()) as ex:
        return list(ex.map(one, ids))
