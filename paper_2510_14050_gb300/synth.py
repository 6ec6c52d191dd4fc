"""Seeded synthetic packet windows (Python side of ``csrc/synth.c``).

The generator is shared by the oracle tests, the GPU tests and the bench, and
holds none of the method's arithmetic.  The five workloads stand in for the
Graph Challenge's synthetic 2^30-packet data set (Sec. V "Dataset"):

=====  =====================================================================
cfg    windows
=====  =====================================================================
1      1 x 2^17 packets; src, dst iid Zipf(1.2) over 2^16 ranks
2      64 x 2^17; src Zipf(1.1)/2^20, dst Zipf(1.3)/2^22; 5% in bursts of 2..100
3      1024 windows, P = floor(2^(10+10u)) in [2^10, 2^20]; heavy hitter (10%),
       scanners (<=10%, fan-out loguniform 16..2^16), rest Zipf(1.1)/2^24
4      8192 x 2^17 (2^30 packets); src, dst Zipf(1.05) over the full 2^32 space
5      serving: P uniform in [2^12, 2^17], traffic as cfg 2, Poisson arrivals
=====  =====================================================================

Ranks map to addresses by ``(k - 1) * 0x9E3779B1 mod 2^32``.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import buildlib

DEFAULT_NWIN = {1: 1, 2: 64, 3: 1024, 4: 8192, 5: 20000}

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = buildlib.build_synth()
        lib = C.CDLL(str(path))
        u64, u64p, u32p = C.c_uint64, C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)
        lib.synth_window_sizes.argtypes = [C.c_int, u64, u64, u64, u64p]
        lib.synth_fill.argtypes = [C.c_int, u64, u64, u64, u64p, u32p, u32p, C.c_int]
        lib.synth_zipf_ranks.argtypes = [C.c_double, u64, u64, u64, u64p]
        lib.synth_arrivals.argtypes = [u64, C.c_double, u64, C.POINTER(C.c_double)]
        for f in (lib.synth_window_sizes, lib.synth_fill, lib.synth_zipf_ranks, lib.synth_arrivals):
            f.restype = C.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


@dataclass
class Windows:
    """Packet windows stored as one stream: window w is [offsets[w], offsets[w+1])."""
    src: np.ndarray      # uint32[total]
    dst: np.ndarray      # uint32[total]
    offsets: np.ndarray  # uint64[nwin + 1], offsets[0] == 0

    @property
    def nwin(self) -> int:
        return len(self.offsets) - 1

    @property
    def total(self) -> int:
        return int(self.offsets[-1])

    def window(self, w: int):
        a, b = int(self.offsets[w]), int(self.offsets[w + 1])
        return self.src[a:b], self.dst[a:b]

    def subset(self, first: int, count: int) -> "Windows":
        a, b = int(self.offsets[first]), int(self.offsets[first + count])
        return Windows(self.src[a:b], self.dst[a:b], self.offsets[first:first + count + 1] - a)


def window_sizes(cfg: int, nwin: int, seed: int = 0, first_window: int = 0) -> np.ndarray:
    out = np.empty(nwin, dtype=np.uint64)
    rc = _load().synth_window_sizes(cfg, seed, first_window, nwin, _ptr(out, C.c_uint64))
    if rc != 0:
        raise ValueError(f"synth_window_sizes failed for cfg {cfg} ({rc})")
    return out


def generate(cfg: int, nwin: int | None = None, seed: int = 0, first_window: int = 0,
             sizes=None, threads: int | None = None, out=None) -> Windows:
    """Windows [first_window, first_window + nwin) of config ``cfg``.

    ``sizes`` overrides the config's window sizes (the traffic model stays the
    config's).  ``out`` may supply preallocated (src, dst) arrays, e.g. pinned
    host memory viewed as numpy."""
    if nwin is None:
        nwin = DEFAULT_NWIN[cfg] if sizes is None else len(sizes)
    if sizes is None:
        sizes = window_sizes(cfg, nwin, seed, first_window)
    sizes = np.asarray(sizes, dtype=np.uint64)
    offsets = np.zeros(nwin + 1, dtype=np.uint64)
    np.cumsum(sizes, out=offsets[1:])
    total = int(offsets[-1])
    if out is None:
        src = np.empty(total, dtype=np.uint32)
        dst = np.empty(total, dtype=np.uint32)
    else:
        src, dst = out
        assert src.dtype == np.uint32 and dst.dtype == np.uint32 and len(src) >= total and len(dst) >= total
    if threads is None:
        threads = max(1, min(os.cpu_count() or 1, 64))
    if total:
        rc = _load().synth_fill(cfg, seed, first_window, nwin, _ptr(offsets, C.c_uint64),
                                _ptr(src, C.c_uint32), _ptr(dst, C.c_uint32), threads)
        if rc != 0:
            raise RuntimeError(f"synth_fill failed for cfg {cfg} ({rc})")
    return Windows(src[:total], dst[:total], offsets)


def zipf_ranks(s: float, n: int, count: int, seed: int = 0) -> np.ndarray:
    out = np.empty(count, dtype=np.uint64)
    if _load().synth_zipf_ranks(s, n, seed, count, _ptr(out, C.c_uint64)) != 0:
        raise ValueError("bad Zipf parameters")
    return out


def arrivals(rate: float, n: int, seed: int = 0) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    if _load().synth_arrivals(seed, rate, n, _ptr(out, C.c_double)) != 0:
        raise ValueError("rate must be positive")
    return out


def rank_to_addr(k):
    k = np.asarray(k, dtype=np.uint64)
    return ((k - np.uint64(1)) * np.uint64(0x9E3779B1) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
