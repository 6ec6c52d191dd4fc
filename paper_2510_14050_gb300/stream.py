"""Out-of-core ingest: windows held in host memory, more of them than the
device budget holds at once, analysed batch by batch with the host-to-device
copy of the next batch overlapped with the analysis of the current one.

This is the paper's sub-partitioning into b_n batches (Sec. III-C) in the
other direction: there, a device's partition is split so that each batch
fits; here the host stream is split into batches of at most
``batch_packets`` packets (whole windows; a larger window forms a batch of
its own).  Two slots -- each a library context with its own CUDA stream,
device input buffers and pinned staging buffers -- alternate: while one
slot's batch is analysed, the other slot's next batch is staged and copied.
Each batch yields its windows' nine quantities; with ``want_sum`` the time
sum of all windows (Table I: A_t summed over t) is kept on the device and
folded batch by batch (``ans_sum_windows``).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import ans


def plan_batches(offsets: np.ndarray, batch_packets: int) -> list[tuple[int, int]]:
    """Consecutive window ranges [w0, w1) of at most batch_packets packets
    each (a window larger than that alone)."""
    offsets = np.asarray(offsets, dtype=np.uint64)
    nwin = len(offsets) - 1
    out = []
    w0 = 0
    while w0 < nwin:
        w1 = w0 + 1
        while w1 < nwin and int(offsets[w1 + 1] - offsets[w0]) <= batch_packets:
            w1 += 1
        out.append((w0, w1))
        w0 = w1
    return out


@dataclass
class StreamResult:
    quantities: np.ndarray  # [nwin, 9] uint64, in window order
    sum: "ans.Matrix | None"  # the time sum of every window (device-resident), or None
    batches: int
    seconds: float
    # per batch (slot, H2D start, H2D end, analysis end) in ms from the first
    # batch's H2D start, from CUDA events on the slots' streams
    timeline: list | None = None


def stream_windows(src, dst, offsets, batch_packets: int = 1 << 24,
                   want_sum: bool = True, device: int = 0, budget_bytes: int = 0,
                   tuning: dict | None = None) -> StreamResult:
    """Analyse every window [offsets[w], offsets[w+1]) of the host arrays
    src/dst in batches of at most batch_packets packets, two batches in
    flight.  src/dst: uint32 numpy arrays (staged through pinned buffers) or
    pinned int32 CPU tensors (copied to the device directly).  ``tuning``:
    launch shapes and paths for both slots' contexts (ans_set_tuning fields).
    Returns the quantities of every window and, with want_sum, their time
    sum, with a per-batch timeline of the copies and the analysis."""
    import time

    import torch

    offsets = np.ascontiguousarray(np.asarray(offsets, dtype=np.uint64))
    nwin = len(offsets) - 1
    pinned = hasattr(src, "is_pinned") and src.is_pinned() and dst.is_pinned()
    if not pinned:
        src = np.ascontiguousarray(src, dtype=np.uint32)
        dst = np.ascontiguousarray(dst, dtype=np.uint32)
    plan = plan_batches(offsets, batch_packets)
    cap = max([int(offsets[b] - offsets[a]) for a, b in plan] + [1])
    cap_w = max([b - a for a, b in plan] + [1])
    dev = f"cuda:{device}"
    slots = []
    for _ in range(2):
        slots.append({
            "ctx": ans.Context(device, budget_bytes=budget_bytes),
            "stream": torch.cuda.Stream(device=device),
            "src": torch.empty(cap, dtype=torch.int32, device=dev),
            "dst": torch.empty(cap, dtype=torch.int32, device=dev),
            "h_src": None if pinned else torch.empty(cap, dtype=torch.int32).pin_memory(),
            "h_dst": None if pinned else torch.empty(cap, dtype=torch.int32).pin_memory(),
            "q": torch.empty((cap_w, 9), dtype=torch.int64, device=dev),
            "h_q": torch.empty((cap_w, 9), dtype=torch.int64).pin_memory(),
            "done": None, "pending": None,
        })
        if tuning:
            slots[-1]["ctx"].set_tuning(**tuning)
    marks = []  # per batch: (slot, H2D start, H2D end, analysis end) events
    quant = np.zeros((nwin, 9), dtype=np.uint64)
    # Batch sums wait in a list and are folded kFold at a time into one
    # (one time-sum call: merge rounds over their sorted links and one column
    # pass), and the rest at the end; a link is re-merged O(log_kFold batches)
    # times and at most kFold + 1 partial sums are held.
    kFold = 8
    partials: list["ans.Matrix"] = []
    retired: list["ans.Matrix"] = []  # merged inputs, freed once later work has passed them
    t0 = time.perf_counter()

    def finish(slot):
        """Collect a slot's previous batch: its quantities and its sum."""
        if slot["pending"] is None:
            return
        (w0, w1), bsum = slot["pending"]
        slot["done"].synchronize()
        for m in retired:
            m.free()
        retired.clear()
        quant[w0:w1] = slot["h_q"][: w1 - w0].numpy().view(np.uint64)
        if bsum is not None:
            partials.append(bsum)
            if len(partials) > kFold:
                folded = slot["ctx"].sum_windows(partials, stream=slot["stream"])
                retired.extend(partials)
                partials[:] = [folded]
        slot["pending"] = None

    try:
        for i, (w0, w1) in enumerate(plan):
            slot = slots[i % 2]
            finish(slot)  # the slot's buffers are free again
            p0, p1 = int(offsets[w0]), int(offsets[w1])
            n = p1 - p0
            st = slot["stream"]
            if pinned:
                h_src, h_dst = src[p0:p1], dst[p0:p1]
            else:  # stage into pinned memory (host copy), then copy asynchronously
                slot["h_src"][:n].numpy().view(np.uint32)[:] = src[p0:p1]
                slot["h_dst"][:n].numpy().view(np.uint32)[:] = dst[p0:p1]
                h_src, h_dst = slot["h_src"][:n], slot["h_dst"][:n]
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            with torch.cuda.stream(st):
                e0.record(st)
                slot["src"][:n].copy_(h_src, non_blocking=True)
                slot["dst"][:n].copy_(h_dst, non_blocking=True)
                e1.record(st)
            flags = ans.BATCH_SUM if want_sum else 0
            _, bsum, _ = slot["ctx"].batch_submit(slot["src"], slot["dst"], offsets[w0:w1 + 1] - offsets[w0], flags,
                                                  out=slot["q"], stream=st, want_ticket=False)
            with torch.cuda.stream(st):
                slot["h_q"][: w1 - w0].copy_(slot["q"][: w1 - w0], non_blocking=True)
                e2.record(st)
                ev = torch.cuda.Event()
                ev.record(st)
            marks.append((i % 2, e0, e1, e2))
            slot["done"] = ev
            slot["pending"] = ((w0, w1), bsum)
        for i in range(len(plan), len(plan) + 2):
            finish(slots[i % 2])
        total_sum = None
        if partials:
            mats = list(partials)
            total_sum = mats[0] if len(mats) == 1 else slots[0]["ctx"].sum_windows(mats, stream=slots[0]["stream"])
            if len(mats) > 1:
                retired.extend(mats)
        torch.cuda.synchronize(device)
        for m in retired:
            m.free()
        seconds = time.perf_counter() - t0
        timeline = None
        if marks:
            first = marks[0][1]
            timeline = [(sl, round(first.elapsed_time(a), 3), round(first.elapsed_time(b), 3),
                         round(first.elapsed_time(c), 3)) for sl, a, b, c in marks]
        return StreamResult(quant, total_sum, len(plan), seconds, timeline)
    finally:
        for s in slots:
            s["ctx"].close()
