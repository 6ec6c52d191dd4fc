"""CPU oracle for anonymized network sensing -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct numpy restatement of what the CUDA library
computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it; the product path never does.  It shares no code
with the CUDA path (``paper_2510_14050_gb300``) and imports nothing from it.

Definitions followed (paper: Table I, Sec. IV-B "Data Representation",
Sec. IV-C "Analytics and Operations"):

* Traffic matrix of a window of packets (s_k, d_k):
  A(i, j) = #{k : s_k = i, d_k = j}; row i is a source, column j a
  destination (Table I caption: A_t(i, j) counts packets from source i to
  destination j).
* DCSR(A): nonempty rows ascending (``row_ids``), ``row_ptr`` = exclusive prefix
  of per-row nonzero counts (the paper's ``degrees``, Sec. IV-B), columns
  ascending within a row (``col_ids``, the paper's ``edges``), values A(i, j) as
  uint64 (the paper's ``weights``).  No explicit zeros.
* The nine network quantities (Table I plus the maxima named in Sec. IV-C):
  valid packets N_V = sum A; unique links = #nonzeros; max link packets =
  max A; unique sources = #nonempty rows; max source packets = max row sum;
  max source fan-out = max nonzeros in a row; unique destinations =
  #nonempty columns; max destination packets = max column sum; max
  destination fan-in = max nonzeros in a column.  Maxima of empty sets are 0.
  Table I prints the fan-out/fan-in formulas with the zero-norm outside the
  inner sum, which would make them at most 1; its C++ column (max of
  ``degrees``) fixes the reading used here: the largest per-row (per-column)
  nonzero count.
* Time sum of windows: (sum_t A_t)(i, j) = sum_t A_t(i, j) (Table I caption,
  A_t indexed by time t).

Every value is an exact integer; uint64 arithmetic throughout (numpy's
``add.reduceat`` on uint64 stays in integers).

Parity status: every function here is pinned by ``tests/test_oracle.py``
(hand-worked windows in ``tests/golden/``, O(P^2) brute force, invariants,
closed forms and planted-mistake checks).
"""
from __future__ import annotations

from typing import NamedTuple, Sequence

import numpy as np

QUANTITY_NAMES = (
    "valid_packets",
    "unique_links",
    "max_link_packets",
    "unique_sources",
    "max_source_packets",
    "max_source_fanout",
    "unique_destinations",
    "max_destination_packets",
    "max_destination_fanin",
)

_U32 = np.uint64(0xFFFFFFFF)
_SH = np.uint64(32)


class DCSR(NamedTuple):
    row_ids: np.ndarray  # uint32[R]
    row_ptr: np.ndarray  # uint64[R + 1]
    col_ids: np.ndarray  # uint32[U]
    vals: np.ndarray     # uint64[U]

    @property
    def nrows(self) -> int:
        return len(self.row_ids)

    @property
    def nnz(self) -> int:
        return len(self.col_ids)


def empty_dcsr() -> DCSR:
    return DCSR(np.zeros(0, np.uint32), np.zeros(1, np.uint64), np.zeros(0, np.uint32), np.zeros(0, np.uint64))


def _dcsr_from_sorted_links(keys: np.ndarray, vals: np.ndarray) -> DCSR:
    """Distinct sorted link keys (src << 32 | dst) with their counts -> DCSR."""
    if len(keys) == 0:
        return empty_dcsr()
    rows = (keys >> _SH).astype(np.uint32)
    cols = (keys & _U32).astype(np.uint32)
    row_ids, first = np.unique(rows, return_index=True)  # rows are already sorted
    row_ptr = np.append(first.astype(np.uint64), np.uint64(len(keys)))
    return DCSR(row_ids.astype(np.uint32), row_ptr, cols, vals.astype(np.uint64))


def traffic_matrix(src: np.ndarray, dst: np.ndarray) -> DCSR:
    """A(i, j) = #{k : s_k = i, d_k = j} as DCSR (Table I caption)."""
    src = np.asarray(src, dtype=np.uint32)
    dst = np.asarray(dst, dtype=np.uint32)
    assert src.shape == dst.shape
    keys = (src.astype(np.uint64) << _SH) | dst.astype(np.uint64)
    links, counts = np.unique(keys, return_counts=True)  # library sort as one step
    return _dcsr_from_sorted_links(links, counts.astype(np.uint64))


def link_keys(m: DCSR) -> np.ndarray:
    """src << 32 | dst for every nonzero of a DCSR, in storage order."""
    nnz_per_row = np.diff(m.row_ptr).astype(np.int64)
    rows = np.repeat(m.row_ids.astype(np.uint64), nnz_per_row)
    return (rows << _SH) | m.col_ids.astype(np.uint64)


def network_quantities(m: DCSR) -> dict:
    """The nine quantities of Table I / Sec. IV-C from a DCSR matrix."""
    u = m.nnz
    r = m.nrows
    q = dict.fromkeys(QUANTITY_NAMES, 0)
    if u == 0:
        return q
    vals = m.vals.astype(np.uint64)
    q["valid_packets"] = int(vals.sum(dtype=np.uint64))           # sum_i sum_j A(i,j)
    q["unique_links"] = u                                           # sum_i sum_j |A(i,j)|_0
    q["max_link_packets"] = int(vals.max())                         # max_ij A(i,j)
    q["unique_sources"] = r                                         # sum_i |sum_j A(i,j)|_0
    starts = m.row_ptr[:-1].astype(np.int64)
    row_sums = np.add.reduceat(vals, starts)                        # sum_j A(i,j) per row
    q["max_source_packets"] = int(row_sums.max())
    q["max_source_fanout"] = int(np.diff(m.row_ptr).max())          # max_i sum_j |A(i,j)|_0
    order = np.argsort(m.col_ids, kind="stable")
    cols = m.col_ids[order]
    cvals = vals[order]
    ucols, cstart = np.unique(cols, return_index=True)
    q["unique_destinations"] = len(ucols)                           # sum_j |sum_i A(i,j)|_0
    col_sums = np.add.reduceat(cvals, cstart)                       # sum_i A(i,j) per column
    q["max_destination_packets"] = int(col_sums.max())
    col_nnz = np.diff(np.append(cstart, u))
    q["max_destination_fanin"] = int(col_nnz.max())                 # max_j sum_i |A(i,j)|_0
    return q


def window_quantities(src: np.ndarray, dst: np.ndarray) -> dict:
    return network_quantities(traffic_matrix(src, dst))


def sum_matrices(mats: Sequence[DCSR]) -> DCSR:
    """(sum_t A_t)(i, j) = sum_t A_t(i, j) as DCSR."""
    mats = [m for m in mats if m.nnz]
    if not mats:
        return empty_dcsr()
    keys = np.concatenate([link_keys(m) for m in mats])
    vals = np.concatenate([m.vals.astype(np.uint64) for m in mats])
    order = np.argsort(keys, kind="stable")
    keys = keys[order]
    vals = vals[order]
    links, first = np.unique(keys, return_index=True)
    sums = np.add.reduceat(vals, first)
    return _dcsr_from_sorted_links(links, sums)


def batch(src: np.ndarray, dst: np.ndarray, offsets: np.ndarray, want_sum: bool = True):
    """Per-window DCSRs and quantities of a windowed stream, plus the time sum."""
    offsets = np.asarray(offsets, dtype=np.uint64)
    mats, quants = [], []
    for w in range(len(offsets) - 1):
        a, b = int(offsets[w]), int(offsets[w + 1])
        m = traffic_matrix(src[a:b], dst[a:b])
        mats.append(m)
        quants.append(network_quantities(m))
    total = sum_matrices(mats) if want_sum else None
    return mats, quants, total


def quantities_array(quants: Sequence[dict]) -> np.ndarray:
    """List of quantity dicts -> uint64[n, 9] in QUANTITY_NAMES order."""
    out = np.zeros((len(quants), len(QUANTITY_NAMES)), dtype=np.uint64)
    for i, q in enumerate(quants):
        out[i] = [q[k] for k in QUANTITY_NAMES]
    return out
