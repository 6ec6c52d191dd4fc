"""Continuous-batching server for windows of packet pairs.

Windows arrive on an open-loop schedule (arrival times in seconds).  The
server admits whatever has arrived into the next free slot -- one slot is one
library context with its own CUDA stream and device input buffers -- so
batches overlap on the GPU.  Each batch is one ``ans_batch_submit`` (the nine
quantities of every window plus the batch's time sum).  Admission is by
device-memory budget: a batch is submitted only if the bytes held by all of
the server's contexts plus the bytes the library says the batch would
allocate (``ans_batch_bytes``) stay within the budget; otherwise it waits for
running batches to complete (an admission stall).  Window latency runs from
the window's arrival to its quantities being visible on the host; it includes
moving its packets to the device: by default the windows sit in page-locked
host memory and the batch's kernels read them there
(``ans_batch_submit_windows``, no staging copy); with ``zero_copy=False``
they are staged into a slot's pinned buffer and copied.

Running time sums (Table I: A_t summed over t) are kept resident on the
device per tumbling bucket of the arrival clock (``bucket_seconds``, e.g. one
minute and one hour), and optionally as sliding sums (``sliding``: horizon
and step in seconds): the sum over the newest horizon/step sub-buckets, kept
exact by adding each completed sub-bucket and subtracting the ones that leave
the horizon (``ans_combine``).  ``checkpoint()`` / ``restore()`` save and
reload every resident sum as DCSR arrays (``ans_matrix_import``).  A worker
thread owns them: each bucket holds a few partial sums of geometrically
growing size, and a completed batch's sum is
merged (``ans_sum_windows``) with the newest partial while they are of similar
size, so the resident set stays small and each link is re-merged O(log n)
times.  The worker waits for each merge before the next one, so every output
is sized by its inputs' actual link counts.  ``bucket_sum()`` merges a
bucket's partials into one matrix.
"""
from __future__ import annotations

import queue as _queue
import threading
import time
from dataclasses import dataclass

import numpy as np

from . import ans


@dataclass
class WindowSource:
    """Packets of the windows to serve: window i is [offsets[i], offsets[i+1])
    of (src, dst), uint32 numpy arrays in host memory."""
    src: np.ndarray
    dst: np.ndarray
    offsets: np.ndarray

    def size(self, i: int) -> int:
        return int(self.offsets[i + 1] - self.offsets[i])


@dataclass
class ServeStats:
    latencies_s: np.ndarray
    quantities: np.ndarray          # [n, 9] uint64 per served window, in arrival order
    packets: int
    wall_s: float
    batches: int
    admission_stalls: int
    max_queue: int

    def percentile_ms(self, q: float) -> float:
        return float(np.percentile(self.latencies_s, q) * 1e3) if len(self.latencies_s) else 0.0

    def summary(self) -> dict:
        return {
            "windows": int(len(self.latencies_s)),
            "p50_ms": round(self.percentile_ms(50), 4),
            "p99_ms": round(self.percentile_ms(99), 4),
            "max_ms": round(float(self.latencies_s.max() * 1e3) if len(self.latencies_s) else 0.0, 4),
            "sustained_packets_per_s": self.packets / self.wall_s if self.wall_s > 0 else 0.0,
            "batches": self.batches,
            "admission_stalls": self.admission_stalls,
            "max_queue": self.max_queue,
        }


class SumKeeper:
    """Resident time sums, maintained by a worker thread: tumbling buckets
    per level, and sliding sums over the newest n sub-buckets of a level
    (``sliding``: {level: n}), kept exact by subtracting the sub-buckets that
    leave the horizon (``ans_combine``)."""

    def __init__(self, device: int, budget_bytes: int, sliding=None):
        import torch
        self.torch = torch
        self.device = device
        self.ctx = ans.Context(device, budget_bytes=budget_bytes)
        self.stream = torch.cuda.Stream(device=device)
        self.buckets = {}      # (level, index) -> [(nnz, Matrix)], newest last
        # sliding level -> {"n": sub-buckets per horizon, "cur": newest sub-bucket,
        # "base": sum of the horizon's complete sub-buckets [cur - n + 1, cur - 1]}
        self.slide = {lv: {"n": int(n), "cur": None, "base": None} for lv, n in (sliding or {}).items()}
        self.lock = threading.Lock()
        self.q = _queue.Queue()
        self.error = None
        self.thread = threading.Thread(target=self._run, daemon=True)
        self.thread.start()

    def add(self, keys, batch_sum):
        """Hand a completed batch's sum to its buckets: keys[level] is the
        bucket index at each level."""
        self.q.put((tuple(keys), batch_sum))

    def _run(self):
        self.torch.cuda.set_device(self.device)
        while True:
            # Everything queued so far is handled together: the batch sums
            # bound for one bucket are first summed in one call, so the
            # number of merges follows the worker's wake-ups, not the batches.
            items = [self.q.get()]
            while True:
                try:
                    items.append(self.q.get_nowait())
                except _queue.Empty:
                    break
            try:
                groups = {}
                for item in items:
                    if item is None:
                        continue
                    keys, mat = item
                    # every level holds its own handle to the same batch sum
                    handles = [mat] + [mat.retain() for _ in keys[1:]]
                    for level, (idx, h) in enumerate(zip(keys, handles)):
                        groups.setdefault((level, idx), []).append(h)
                for key, mats in sorted(groups.items()):
                    if len(mats) > 1:
                        merged = self.ctx.sum_windows(mats, stream=self.stream)
                        for m in mats:
                            m.free()
                        self.stream.synchronize()
                        mats = [merged]
                    self._insert(key, mats[0])
                    if key[0] in self.slide:
                        self._advance(key[0], key[1])
            except Exception as e:  # surfaced by drain()
                self.error = e
            finally:
                for _ in items:
                    self.q.task_done()
            if any(item is None for item in items):
                return

    def _insert(self, key, mat):
        with self.lock:
            parts = self.buckets.setdefault(key, [])
            parts.append((mat.nnz, mat))
            while len(parts) >= 2 and parts[-2][0] <= 2 * parts[-1][0]:
                (_, m1), (_, m2) = parts[-2], parts[-1]
                merged = self.ctx.sum_windows([m1, m2], stream=self.stream)
                m1.free()
                m2.free()
                self.stream.synchronize()
                parts[-2:] = [(merged.nnz, merged)]

    def _merged(self, key):
        """The bucket's partials merged into one matrix (kept as its only partial)."""
        parts = self.buckets.get(key)
        if not parts:
            return None
        if len(parts) > 1:
            mats = [m for _, m in parts]
            merged = self.ctx.sum_windows(mats, stream=self.stream)
            for m in mats:
                m.free()
            self.stream.synchronize()
            parts[:] = [(merged.nnz, merged)]
        return parts[0][1]

    def _advance(self, level, idx):
        """Sub-bucket idx of a sliding level received data: once it is newer
        than the current one, fold the completed sub-buckets into the base and
        take out the ones that left the horizon."""
        st = self.slide[level]
        with self.lock:
            if st["cur"] is None:
                st["cur"] = idx
                return
            if idx <= st["cur"]:
                return
            n, cur = st["n"], st["cur"]
            lo_new = idx - n + 1  # oldest sub-bucket of the new horizon
            mats, signs = [], []
            for j in range(max(cur, lo_new), idx):  # completed and still inside
                m = self._merged((level, j))
                if m is not None:
                    mats.append(m)
                    signs.append(1)
            for j in range(cur - n + 1, min(cur, lo_new)):  # in the base, now outside
                m = self._merged((level, j))
                if m is not None:
                    mats.append(m)
                    signs.append(-1)
            if mats:
                if st["base"] is not None:
                    mats.insert(0, st["base"])
                    signs.insert(0, 1)
                new_base = self.ctx.combine(mats, signs, stream=self.stream)
                self.stream.synchronize()
                if st["base"] is not None:
                    st["base"].free()
                st["base"] = new_base
            for j in [k[1] for k in list(self.buckets) if k[0] == level and k[1] < lo_new]:
                for _, m in self.buckets.pop((level, j)):  # sub-buckets that left: no longer needed
                    m.free()
            st["cur"] = idx

    def sliding_sum(self, level):
        """Sum of the windows in the newest n sub-buckets of a sliding level
        (None if it has none)."""
        self.drain()
        st = self.slide[level]
        with self.lock:
            if st["cur"] is None:
                return None
            cur = self._merged((level, st["cur"]))
            mats = [m for m in (st["base"], cur) if m is not None]
            if len(mats) == 1:
                return mats[0].retain()
            out = self.ctx.sum_windows(mats, stream=self.stream)
            self.stream.synchronize()
            return out

    def checkpoint(self, path):
        """Save every resident sum (bucket sums, sliding bases and their
        state) to `path` (.npz) as DCSR arrays."""
        import json
        self.drain()
        arrays, meta = {}, {"buckets": [], "slide": {}}
        with self.lock:
            for i, key in enumerate(sorted(self.buckets)):
                m = self._merged(key)
                for name, a in zip(("row_ids", "row_ptr", "col_ids", "vals"), m.to_numpy()):
                    arrays[f"b{i}_{name}"] = a
                meta["buckets"].append([int(key[0]), int(key[1])])
            for lv, st in self.slide.items():
                meta["slide"][str(lv)] = {"n": st["n"], "cur": st["cur"], "base": st["base"] is not None}
                if st["base"] is not None:
                    for name, a in zip(("row_ids", "row_ptr", "col_ids", "vals"), st["base"].to_numpy()):
                        arrays[f"s{lv}_{name}"] = a
        np.savez(path, meta=np.frombuffer(json.dumps(meta).encode(), dtype=np.uint8), **arrays)

    def restore(self, path):
        """Replace the resident sums by the ones saved by checkpoint()."""
        import json
        self.drain()
        z = np.load(path)
        meta = json.loads(bytes(z["meta"]).decode())
        with self.lock:
            for parts in self.buckets.values():
                for _, m in parts:
                    m.free()
            self.buckets = {}
            for i, (lv, idx) in enumerate(meta["buckets"]):
                m = self.ctx.import_matrix(*(z[f"b{i}_{n}"] for n in ("row_ids", "row_ptr", "col_ids", "vals")))
                self.buckets[(lv, idx)] = [(m.nnz, m)]
            for lv_s, st in meta["slide"].items():
                lv = int(lv_s)
                old = self.slide.get(lv, {}).get("base")
                if old is not None:
                    old.free()
                base = None
                if st["base"]:
                    base = self.ctx.import_matrix(*(z[f"s{lv}_{n}"] for n in ("row_ids", "row_ptr", "col_ids", "vals")))
                self.slide[lv] = {"n": st["n"], "cur": st["cur"], "base": base}

    def drain(self):
        self.q.join()
        if self.error is not None:
            raise self.error

    def bucket_sum(self, key):
        self.drain()
        with self.lock:
            return self._merged(key)

    def memory(self) -> int:
        return self.ctx.memory()[0]

    def close(self):
        self.q.put(None)
        self.thread.join()
        for parts in self.buckets.values():
            for _, m in parts:
                m.free()
        self.buckets = {}
        for st in self.slide.values():
            if st["base"] is not None:
                st["base"].free()
                st["base"] = None
        self.ctx.close()


class Server:
    def __init__(self, device: int = 0, slots: int = 4, budget_bytes: int = 64 << 30,
                 max_batch_windows: int = 256, max_batch_packets: int = 1 << 24,
                 bucket_seconds=(60.0, 3600.0), keep_sums: bool = True, zero_copy: bool = True,
                 sliding=(), tuning: dict | None = None):
        import torch
        self.torch = torch
        self.device = device
        self.max_batch_windows = max_batch_windows
        self.max_batch_packets = max_batch_packets
        self.bucket_seconds = tuple(bucket_seconds)
        # sliding horizons (seconds, step): each adds a level of tumbling
        # sub-buckets of `step` seconds, summed over the newest horizon/step
        self.sliding = tuple((float(h), float(g)) for h, g in sliding)
        self.level_seconds = self.bucket_seconds + tuple(g for _, g in self.sliding)
        self.keep_sums = keep_sums
        self.zero_copy = zero_copy
        self.budget = budget_bytes
        self.slots = []
        for _ in range(slots):
            ctx = ans.Context(device, budget_bytes=budget_bytes)
            if tuning:  # launch shapes and paths (ans_set_tuning fields), e.g. from Context.autotune
                ctx.set_tuning(**tuning)
            st = torch.cuda.Stream(device=device)
            self.slots.append({
                "ctx": ctx, "stream": st,
                "src": torch.empty(max_batch_packets, dtype=torch.int32, device=f"cuda:{device}"),
                "dst": torch.empty(max_batch_packets, dtype=torch.int32, device=f"cuda:{device}"),
                "h_src": torch.empty(max_batch_packets, dtype=torch.int32).pin_memory(),
                "h_dst": torch.empty(max_batch_packets, dtype=torch.int32).pin_memory(),
                "q_dev": torch.empty((max_batch_windows, 9), dtype=torch.int64, device=f"cuda:{device}"),
                "q_host": torch.empty((max_batch_windows, 9), dtype=torch.int64).pin_memory(),
                "inflight": None,
            })
        nb = len(self.bucket_seconds)
        slide = {nb + i: max(1, int(round(h / g))) for i, (h, g) in enumerate(self.sliding)}
        self.sums = SumKeeper(device, budget_bytes, slide) if keep_sums else None
        if self.sums is not None and tuning:
            self.sums.ctx.set_tuning(**tuning)

    def live_bytes(self) -> int:
        """Device bytes held by all of the server's contexts."""
        return sum(s["ctx"].memory()[0] for s in self.slots) + (self.sums.memory() if self.sums else 0)

    def sliding_sum(self, i: int = 0):
        """The time sum of every served window that arrived in the newest
        horizon/step sub-buckets of sliding horizon i (None if none)."""
        return self.sums.sliding_sum(len(self.bucket_seconds) + i) if self.sums else None

    def checkpoint(self, path):
        """Save the resident sums (tumbling buckets, sliding bases) to a file."""
        self.sums.checkpoint(path)

    def restore(self, path):
        """Load resident sums saved by checkpoint() (replacing the current ones)."""
        self.sums.restore(path)

    def bucket_sum(self, level: int, idx: int):
        """One matrix: the time sum of every served window whose arrival falls
        in bucket idx of bucket_seconds[level] (None if there is none)."""
        return self.sums.bucket_sum((level, idx)) if self.sums else None

    def close(self):
        if self.sums is not None:
            self.sums.close()
        for s in self.slots:
            s["ctx"].close()

    def serve(self, source: WindowSource, arrivals: np.ndarray, order=None) -> ServeStats:
        """Serve windows order[k] (default k) arriving at arrivals[k] seconds
        after the start; returns latencies and quantities in arrival order."""
        torch = self.torch
        n = len(arrivals)
        order = np.arange(n) if order is None else np.asarray(order)
        lat = np.zeros(n)
        quants = np.zeros((n, 9), dtype=np.uint64)
        batches = stalls = max_q = 0
        packets = 0
        next_k = 0             # next arrival not yet admitted
        queue = []             # arrived, not yet submitted (indices into arrivals)
        flags = ans.BATCH_SUM if self.keep_sums else 0
        if self.zero_copy:
            # windows arrive in page-locked host memory; the kernels read them there
            pin_src = torch.from_numpy(source.src.view(np.int32)).pin_memory()
            pin_dst = torch.from_numpy(source.dst.view(np.int32)).pin_memory()
        t0 = time.perf_counter()

        def bucket_ids(k):
            return tuple(int(arrivals[k] // w) for w in self.level_seconds)

        def complete(slot):
            nonlocal packets
            job = slot["inflight"]
            slot["inflight"] = None
            job["event"].synchronize()
            t_done = time.perf_counter() - t0
            qh = slot["q_host"][: len(job["ks"])].numpy().view(np.uint64)
            for j, k in enumerate(job["ks"]):
                lat[k] = t_done - arrivals[k]
                quants[k] = qh[j]
            packets += job["packets"]
            if job["sum"] is not None:
                self.sums.add(job["buckets"], job["sum"])

        def batch_offsets(ks):
            offs = np.zeros(len(ks) + 1, dtype=np.uint64)
            np.cumsum([source.size(int(order[k])) for k in ks], out=offs[1:])
            return offs

        def submit(slot, ks, offs):
            ctx, st = slot["ctx"], slot["stream"]
            if self.zero_copy:
                wins = []
                for k in ks:
                    w = int(order[k])
                    a, b = int(source.offsets[w]), int(source.offsets[w + 1])
                    wins.append((pin_src.data_ptr() + 4 * a, pin_dst.data_ptr() + 4 * a, b - a))
                with torch.cuda.stream(st):
                    _, summ, _ = ctx.batch_submit_windows(wins, flags, out=slot["q_dev"], stream=st,
                                                          want_ticket=False)
                    slot["q_host"][: len(ks)].copy_(slot["q_dev"][: len(ks)], non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(st)
                slot["inflight"] = {"ks": list(ks), "event": ev, "sum": summ, "packets": int(offs[-1]),
                                    "buckets": bucket_ids(ks[0])}
                return
            hs, hd = slot["h_src"].numpy().view(np.uint32), slot["h_dst"].numpy().view(np.uint32)
            for j, k in enumerate(ks):
                w = int(order[k])
                a, b = int(source.offsets[w]), int(source.offsets[w + 1])
                hs[int(offs[j]):int(offs[j + 1])] = source.src[a:b]
                hd[int(offs[j]):int(offs[j + 1])] = source.dst[a:b]
            pos = int(offs[-1])
            with torch.cuda.stream(st):
                slot["src"][:pos].copy_(slot["h_src"][:pos], non_blocking=True)
                slot["dst"][:pos].copy_(slot["h_dst"][:pos], non_blocking=True)
                _, summ, _ = ctx.batch_submit(slot["src"], slot["dst"], offs, flags, out=slot["q_dev"],
                                              stream=st, want_ticket=False)
                slot["q_host"][: len(ks)].copy_(slot["q_dev"][: len(ks)], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(st)
            slot["inflight"] = {"ks": list(ks), "event": ev, "sum": summ, "packets": pos,
                                "buckets": bucket_ids(ks[0])}

        stalled_head = -1
        while True:
            now = time.perf_counter() - t0
            while next_k < n and arrivals[next_k] <= now:
                queue.append(next_k)
                next_k += 1
            max_q = max(max_q, len(queue))
            progressed = False
            for slot in self.slots:
                job = slot["inflight"]
                if job is not None and job["event"].query():
                    complete(slot)
                    progressed = True
            for slot in self.slots:
                if not queue:
                    break
                if slot["inflight"] is not None:
                    continue
                # continuous batching: take what has arrived, one time bucket per batch
                ks, pk = [], 0
                b0 = bucket_ids(queue[0])
                for k in queue:
                    sz = source.size(int(order[k]))
                    if ks and (len(ks) >= self.max_batch_windows or pk + sz > self.max_batch_packets
                               or bucket_ids(k) != b0):
                        break
                    ks.append(k)
                    pk += sz
                offs = batch_offsets(ks)
                need = slot["ctx"].batch_bytes(offs, flags)
                if self.live_bytes() + need > self.budget:
                    if stalled_head != ks[0]:
                        stalls += 1
                        stalled_head = ks[0]
                    if all(s["inflight"] is None for s in self.slots):
                        if self.sums is not None:
                            self.sums.drain()  # merges may still release memory
                            if self.live_bytes() + need <= self.budget:
                                continue
                        raise RuntimeError(f"a batch of {len(ks)} windows needs {need} bytes and does not fit in "
                                           f"the {self.budget}-byte budget with nothing running")
                    break  # wait for running batches to release memory
                submit(slot, ks, offs)
                del queue[: len(ks)]
                batches += 1
                progressed = True
            if next_k >= n and not queue and all(s["inflight"] is None for s in self.slots):
                break
            if not progressed:
                if next_k < n and not queue:
                    wait = arrivals[next_k] - (time.perf_counter() - t0)
                    if wait > 2e-4:
                        time.sleep(min(wait - 1e-4, 2e-3))
                else:
                    time.sleep(2e-5)
        wall = time.perf_counter() - t0
        torch.cuda.synchronize(self.device)
        return ServeStats(latencies_s=lat, quantities=quants, packets=packets, wall_s=wall, batches=batches,
                          admission_stalls=stalls, max_queue=max_q)


def pool_source(nwin: int, seed: int = 0) -> WindowSource:
    """A pool of serving-size windows: P uniform in [2^12, 2^17], traffic as
    the 64-window batch (Zipf sources/destinations, 5% bursts)."""
    from . import synth
    w = synth.generate(5, nwin=nwin, seed=seed)
    return WindowSource(w.src, w.dst, w.offsets)


def poisson_schedule(rate: float, n: int, pool: int, seed: int = 0):
    """Arrival times (s) of n windows at `rate` windows/s, and which pool
    window each one carries."""
    from . import synth
    t = synth.arrivals(rate, n, seed=seed)
    order = (np.arange(n) * 7919) % pool
    return t, order
