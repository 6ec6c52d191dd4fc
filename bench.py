#!/usr/bin/env python3
"""Throughput of the batched anonymized-network-sensing path on GB300.

One step = one pass of the whole hot path over one batch of synthetic
windows: pack + sort + run-length reduction of every window, the nine
quantities of every window, and the time sum of all windows of the batch
(its DCSR and quantities).  The default workload is the 2^30-packet
aggregate: 8192 windows of 2^17 packets, src and dst Zipf(1.05) over the full
2^32 address space, per-window quantities plus the single summed matrix.
The 64-window workload (--config 2) also returns every window's DCSR.

Prints ONE JSON line (rank 0).  Fields beyond the base contract:
  roofline       the whole step's algorithmic bytes (read every packet pair
                 once, write the quantities, write the DCSR that is returned)
                 over the step time, against the measured HBM copy bandwidth;
                 extra passes of the method are not credited
  kernel_roofline  the dominant kernel: its own algorithmic bytes per launch
                 (e.g. 16 B per key per digit pass) over its mean launch time
  per_window     the plain method: one ans_build_window per window + one
                 ans_sum_windows
  cpu_baseline   the CPU oracle on this host: every core (a process per core,
                 windows split between them) on a bounded sample, and one
                 core
`--impl reference` times the CPU oracle instead (the reference arm).
Multi-GPU (torchrun): independent replicas, one batch of distinct windows per
rank, barrier + max-over-ranks timing, weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "packets/s (batched hot path: per-window quantities + time-summed DCSR)"
UNIT = "packets/s"
FLUSH_BYTES = 512 << 20  # > 129 MB L2
FALLBACK_HBM_GBS = 6800.0

WORKLOADS = {
    1: "1 window x 2^17 packets; src, dst Zipf(1.2)/2^16; DCSR + 9 quantities + its time sum",
    2: "64 windows x 2^17 packets (8.4M pairs); src Zipf(1.1)/2^20, dst Zipf(1.3)/2^22, 5% bursts of 2..100; "
       "per-window DCSR + 9 quantities + 64-window time sum",
    3: "1024 windows, P loguniform [2^10, 2^20]; heavy hitter 10%, scanners, rest Zipf(1.1)/2^24; "
       "per-window 9 quantities + time-summed DCSR",
    4: "2^13 windows x 2^17 (2^30 pairs, 8 GiB); src, dst Zipf(1.05) over 2^32; per-window 9 quantities + "
       "one time-summed DCSR",
}
DEFAULT_CONFIG = 4
DEFAULT_NWIN = {1: 1, 2: 64, 3: 1024, 4: 8192}
# Per-window DCSR matrices are returned on the small workloads; on the large
# ones the step returns the windows' quantities and the summed matrix.
WANT_MATRICES = {1: True, 2: True, 3: False, 4: False}
# Windows of the oracle's bounded samples: all cores (a process per core) and
# the reference arm's per-step sample.
ORACLE_SAMPLE = {1: 1, 2: 64, 3: 192, 4: 512}
REFERENCE_SAMPLE = {1: 1, 2: 64, 3: 96, 4: 256}

# DRAM traffic per packet (ncu dram__bytes_read.sum + dram__bytes_write.sum),
# from a capture of a smaller case of the same workload (2^25 packets: 256
# windows of 2^17, inputs and scratch well above L2): `step` sums every
# library kernel of one step, `kernels` gives the bytes per launch of a
# kernel family.  Scaled to the bench's workload by its packet count (the
# kernels stream their data, so traffic grows with the packets).  Valid only
# for the library sources it was captured with and the paths and launch
# shapes that decide the traffic (else the bench reports null).
NCU_TRAFFIC = {
    4: {"library": "aa3d1cc8fee92455", "matrices": False,
        "paths": {"agg_path": 3, "sum_path": 2, "col_hash": 1, "key_threads": 256, "key_blocks": 4},
        "step": 365.65, "kernels": {"onesweep_pk": 19.74, "regroup": 19.73, "rle": 23.18}},
}


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", type=int, default=DEFAULT_CONFIG, choices=sorted(WORKLOADS))
    ap.add_argument("--nwin", type=int, default=None, help="override the number of windows per step")
    ap.add_argument("--impl", default="ans", choices=["ans", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-per-window", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-kernel-timing", action="store_true")
    ap.add_argument("--matrices", type=int, default=None, choices=[0, 1],
                    help="return per-window DCSR matrices (default: 1 on configs 1-2, 0 on 3-4)")
    ap.add_argument("--tuning", default=None,
                    help="fix launch shapes and paths instead of autotuning, e.g. key=512,0,2;kv=512,0,1;agg_path=1")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--stream-batches", type=int, default=4,
                    help="out-of-core run: the step's windows streamed from pinned host memory in this many "
                         "batches, two in flight (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=1e4, help="serving arrivals, windows/s")
    ap.add_argument("--serve-windows", type=int, default=20000)
    ap.add_argument("--serve-budget-gib", type=float, default=64.0)
    ap.add_argument("--serve-batch-windows", type=int, default=256, help="most windows in one serving batch")
    ap.add_argument("--serve-batch-packets", type=int, default=1 << 24, help="most packets in one serving batch")
    ap.add_argument("--serve-no-autotune", action="store_true",
                    help="serve with the library's default launch shapes and paths")
    ap.add_argument("--serve-sweep", action="store_true",
                    help="only serving: every rate of 1e3..1e5 windows/s x budgets 32/64/128 GiB, one line each")
    ap.add_argument("--library-sort", action="store_true",
                    help="also time a library radix sort (torch.sort: CUB) of the step's packed 64-bit keys")
    return ap.parse_args(argv)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def host_cpu():
    """(logical cores this process may use, CPU model name)."""
    try:
        cores = len(os.sched_getaffinity(0))
    except Exception:
        cores = os.cpu_count() or 1
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu model")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return cores, model or "unknown"


def library_fingerprint() -> str:
    """Hash of the CUDA library's code (kernels and launchers): comments and
    blank lines are left out, so that a change of wording keeps it."""
    import re
    h = hashlib.sha256()
    csrc = Path(ROOT) / "paper_2510_14050_gb300" / "csrc"
    for p in sorted(csrc.glob("ans_*.cu")) + sorted(csrc.glob("*.cuh")):
        text = re.sub(r"/\*.*?\*/", "", p.read_text(), flags=re.S)
        lines = [re.sub(r"\s*//.*$", "", ln).rstrip() for ln in text.splitlines()]
        h.update(p.name.encode())
        h.update("\n".join(ln for ln in lines if ln).encode())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clock/throttle samples taken during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def algorithmic_bytes(sizes, quants, sum_q, with_matrices: bool):
    """Bytes the method must move in one step: every packet pair read once
    (8 B), the nine quantities written (72 B per window), each returned DCSR
    written once (12 B per link: column id + count; 12 B per row: row id +
    row pointer; 8 B for the closing row pointer).  Extra passes of the
    method are not credited."""
    b = 0
    for p, q in zip(sizes, quants):
        b += 8 * int(p) + 72
        if with_matrices:
            b += 12 * q["unique_links"] + 12 * q["unique_sources"] + 8
    if sum_q is not None:
        b += 12 * sum_q["unique_links"] + 12 * sum_q["unique_sources"] + 8 + 72
    return b


def kernel_bytes_per_step(name, sizes, quants, sum_q, tuning, with_matrices):
    """Algorithmic bytes one step's launches of kernel family `name` move:
    reads + writes each item needs once per pass.  P = packets (split by
    window-sort path), U/R = links/rows of the windows, Us/Rs = links/rows of
    the time sum."""
    cluster_max = 1 << 17
    on_chip = bool(tuning) and tuning.get("win_path") == 0
    p_cl = sum(int(p) for p in sizes if on_chip and p <= cluster_max)
    p_all = sum(int(p) for p in sizes)
    p_os = p_all - p_cl
    u = sum(q["unique_links"] for q in quants)
    r = sum(q["unique_sources"] for q in quants)
    us = sum_q["unique_links"] if sum_q else 0
    rs = sum_q["unique_sources"] if sum_q else 0
    rounds = max(1, (len(sizes) - 1).bit_length()) if len(sizes) > 1 else 0
    # the windows' order from the packet sort: the packets carry 16-bit window ids
    regroup = bool(tuning) and tuning.get("agg_path") == 3 and sum_q is not None and 2 <= len(sizes) <= 1 << 16
    rules = {
        "pack_hist": 16 * p_os,                        # read pairs, write keys
        "onesweep": 8 * 16 * p_os,                     # 8 passes: read + write a key
        "cluster_sort": 16 * p_cl,                     # read pairs, write sorted keys
        "hash_insert": 8 * p_all,                      # read pairs
        "hash_compact": 32 * u,                        # slot in, (key, count) out
        "onesweep_hash": 8 * 32 * u,                   # 8 passes over (key, count)
        "rle": 8 * p_all + 12 * u + 20 * r + 8 * u + 12 * us + 20 * rs,
        "finish": 32 * u + 32 * r + 28 * us + 32 * rs,
        "onesweep_col": 4 * 16 * u + 4 * 16 * us,      # (dst, u32 count) per digit pass
        "colhash": 8 * u,
        "colstat": 8 * u + 8 * us,
        "gather": 28 * u,                              # link + its row in, (key, count) out
        "merge": rounds * 32 * u,                      # each round: read both runs, write the merge
        "onesweep_sum": 8 * 32 * u,                    # 8 passes over (key, count)
        "scan_u64": 16 * us,
        "pack_hist_sum": 16 * p_all,                   # the time sum's packets: read pairs, write keys
        "onesweep_pk": 8 * (20 if regroup else 16) * p_all,  # 8 passes over the batch's packets (+ window ids)
        "wid_fill": 2 * p_all,                         # a window id per packet
        "regroup": 20 * p_all + 18 * p_all,            # (id, key) in and out; then (id, key) in, key out
        "colhash_part": 24 * u,                        # regroup (read twice, write) + count (read) per link
        "hq_split": 24 * p_all,                        # regroup packets: read twice, write once
        "hq_links": 8 * p_all + 12 * u,                # read packets, append distinct links
        "hq_keysplit": 2 * 3 * 8 * u,                  # two stages: read links twice, write once
        "hq_keyhash": 2 * 8 * u,                       # two stages: read links
    }
    return rules.get(name)


# ---- the CPU oracle, for the baseline and the reference arm -----------------
# A process per core; the windows of the sample are split between them in
# contiguous ranges.  Each process builds its windows' matrices and
# quantities and the time sum of its range; the parent adds the ranges' sums
# (the time sum is associative: Table I's A_t added link by link).

def _oracle_range(args):
    path_src, path_dst, offsets, lo, hi = args
    import oracle
    src = np.load(path_src, mmap_mode="r")
    dst = np.load(path_dst, mmap_mode="r")
    mats = []
    for i in range(lo, hi):
        a, b = int(offsets[i]), int(offsets[i + 1])
        m = oracle.traffic_matrix(np.asarray(src[a:b]), np.asarray(dst[a:b]))
        oracle.network_quantities(m)
        mats.append(m)
    return tuple(oracle.sum_matrices(mats))


def _oracle_warm(_):
    import oracle  # noqa: F401  (the import is the warm-up)
    time.sleep(0.2)
    return os.getpid()


class OraclePool:
    """The oracle over a sample of windows on every host core."""

    def __init__(self, w, cores: int):
        import multiprocessing as mp
        self.w = w
        self.cores = max(1, cores)
        self.dir = tempfile.TemporaryDirectory(prefix="ans_oracle_")
        self.paths = (os.path.join(self.dir.name, "src.npy"), os.path.join(self.dir.name, "dst.npy"))
        np.save(self.paths[0], w.src)
        np.save(self.paths[1], w.dst)
        # spawn: the parent holds a CUDA context, which a forked child must not inherit
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.pool.map(_oracle_warm, range(self.cores), chunksize=1)  # every worker up, numpy imported

    def run(self):
        """One pass over the sample; returns (packets, seconds)."""
        import oracle
        n = self.w.nwin
        cuts = np.linspace(0, n, min(self.cores, n) + 1).astype(int)
        jobs = [(*self.paths, self.w.offsets, int(a), int(b)) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
        t0 = time.perf_counter()
        parts = [oracle.DCSR(*p) for p in self.pool.map(_oracle_range, jobs, chunksize=1)]
        oracle.network_quantities(oracle.sum_matrices(parts))
        return self.w.total, time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()
        self.dir.cleanup()


def time_oracle_one_core(w, budget_s=5.0):
    """The oracle over windows of `w` on one core until ~budget_s has elapsed
    (at least one window) plus their time sum; (packets/s, windows, s)."""
    import oracle
    t0 = time.perf_counter()
    mats, pk, n = [], 0, 0
    for i in range(w.nwin):
        s, d = w.window(i)
        m = oracle.traffic_matrix(s, d)
        oracle.network_quantities(m)
        mats.append(m)
        pk += len(s)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    oracle.network_quantities(oracle.sum_matrices(mats))
    dt = time.perf_counter() - t0
    return pk / dt, n, dt


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2510_14050_gb300 import synth
    nwin = args.nwin or DEFAULT_NWIN[args.config]
    sample = max(1, min(nwin, REFERENCE_SAMPLE[args.config]))
    w = synth.generate(args.config, nwin=sample)
    cores, model = host_cpu()
    pool = OraclePool(w, cores)
    try:
        for _ in range(args.warmup):
            pool.run()
        total_s = 0.0
        for _ in range(args.steps):
            _, dt = pool.run()
            total_s += dt
    finally:
        pool.close()
    value = w.total * args.steps / total_s
    sample_desc = (f"first {sample} of {nwin} windows ({w.total} packets) + their time sum per step; "
                   f"numpy oracle, a process per core over windows ({cores} cores, {model})")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_s / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.config], "sample": sample_desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample_desc,
                         "cpu_model": model},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def serving_tuning(local, pool, nwin=256):
    """Launch shapes and paths for the server's contexts: the autotuner's
    choice on a batch of the first `nwin` pool windows with a time sum."""
    import torch

    from paper_2510_14050_gb300 import ans
    n = int(pool.offsets[min(nwin, pool.offsets.size - 1)])
    src = torch.from_numpy(pool.src[:n].view(np.int32)).cuda(local)
    dst = torch.from_numpy(pool.dst[:n].view(np.int32)).cuda(local)
    ctx = ans.Context(local)
    try:
        return ctx.autotune(src, dst, pool.offsets[: min(nwin, pool.offsets.size - 1) + 1], flags=ans.BATCH_SUM)
    finally:
        ctx.close()


def run_serving(local, rate, n, budget_gib, pool=None, seed=0, tuning=None, batch_windows=256,
                batch_packets=1 << 24):
    """Open-loop Poisson arrivals of serving-size windows (P uniform in
    [2^12, 2^17], traffic as the 64-window batch) through the
    continuous-batching server; latency from arrival to quantities on the host,
    H2D included.  Running 1-minute and 1-hour tumbling sums stay resident."""
    from paper_2510_14050_gb300 import serve
    pool = pool or serve.pool_source(512, seed=seed)
    npool = pool.offsets.size - 1
    srv = serve.Server(device=local, slots=4, budget_bytes=int(budget_gib * (1 << 30)),
                       max_batch_windows=batch_windows, max_batch_packets=batch_packets,
                       bucket_seconds=(60.0, 3600.0), tuning=tuning)
    try:
        warm_t, warm_o = serve.poisson_schedule(rate, min(n, 200), npool, seed=seed + 1)
        srv.serve(pool, warm_t, warm_o)
        arr, order = serve.poisson_schedule(rate, n, npool, seed=seed)
        st = srv.serve(pool, arr, order)
        out = {"lambda_windows_per_s": rate, "budget_gib": budget_gib, "slots": 4,
               "max_batch_windows": batch_windows, "max_batch_packets": batch_packets,
               "tuned": bool(tuning), **st.summary(),
               "offered_packets_per_s": float(np.diff(pool.offsets)[order].sum() / max(arr[-1], 1e-9))}
    finally:
        srv.close()
    return out, pool


def parse_tuning(text: str) -> dict:
    kw = {}
    for part in text.split(";"):
        fam, vals = part.split("=")
        fam = fam.strip()
        if fam.endswith("_path") or fam in ("col_hash", "merge_tile"):  # e.g. agg_path=1; graph_path=0 sets graph
            kw["graph" if fam == "graph_path" else fam] = int(vals)
            continue
        for field, v in zip(("threads", "rank", "blocks"), vals.split(",")):
            kw[f"{fam}_{field}"] = int(v)
    return kw


def main(argv=None):
    args = parse_args(argv)
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    from paper_2510_14050_gb300 import ans, replicas, synth

    torch.cuda.set_device(local)
    if args.serve_sweep:
        if rank == 0:
            from paper_2510_14050_gb300 import serve
            pool = serve.pool_source(512, seed=0)
            tun = None if args.serve_no_autotune else serving_tuning(local, pool)
            for budget in (32.0, 64.0, 128.0):
                for rate in (1e3, 3e3, 1e4, 3e4, 1e5):
                    n = max(args.serve_windows, int(min(rate * 10.0, 200000)))
                    res, pool = run_serving(local, rate, n, budget, pool, tuning=tun,
                                            batch_windows=args.serve_batch_windows,
                                            batch_packets=args.serve_batch_packets)
                    print(json.dumps({"metric": "serving window latency", "unit": "ms", **res}), flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x: float) -> float:
        return replicas.max_over_ranks(x, dist, "cuda")

    cfg = args.config
    nwin = args.nwin or DEFAULT_NWIN[cfg]
    with_mats = bool(WANT_MATRICES[cfg] if args.matrices is None else args.matrices)
    flags = ans.BATCH_SUM | (ans.BATCH_MATRICES if with_mats else 0)
    t_gen = time.perf_counter()
    w = synth.generate(cfg, nwin=nwin, first_window=replicas.first_window(rank, nwin))
    t_gen = time.perf_counter() - t_gen
    total = w.total
    sizes = np.diff(w.offsets)

    ctx = ans.Context(local)
    stream = torch.cuda.current_stream()
    src_h = torch.from_numpy(w.src.view(np.int32)).pin_memory()
    dst_h = torch.from_numpy(w.dst.view(np.int32)).pin_memory()
    src_d = src_h.cuda()
    dst_d = dst_h.cuda()
    q_dev = torch.zeros((nwin, 9), dtype=torch.int64, device="cuda")
    q_host = torch.zeros((nwin, 9), dtype=torch.int64).pin_memory()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def step(s, d):
        mats, summ, _ = ctx.batch_submit(s, d, w.offsets, flags, out=q_dev, want_ticket=False)
        return mats, summ

    def release(res):
        mats, summ = res
        for m in mats or ():
            m.free()
        summ.free()

    tuning = None
    t_tune = time.perf_counter()
    if args.tuning:
        ctx.set_tuning(**parse_tuning(args.tuning))
        tuning = ctx.get_tuning()
    elif not args.no_autotune:
        tuning = ctx.autotune(src_d, dst_d, w.offsets, flags=flags)
    t_tune = time.perf_counter() - t_tune
    for _ in range(max(args.warmup, 0)):
        res = step(src_d, dst_d)
        torch.cuda.synchronize()
        release(res)
    if tuning is None:
        tuning = ctx.get_tuning()
    quants = ans.quantities_from_tensor(q_dev)
    res = step(src_d, dst_d)
    torch.cuda.synchronize()
    sum_q = res[1].quantities()
    release(res)
    alg_bytes = algorithmic_bytes(sizes, quants, sum_q, with_mats)

    # ---- timed region: device-resident inputs, the production path (each
    # batch's launch sequence replayed as a CUDA graph), no per-kernel events.
    # A step's results are released after its end event has been recorded
    # (the release waits for the step, outside the step's own event pair).
    clocks = ClockSampler(local)
    barrier()
    clocks.start()

    def timed_steps(fn, k, per_kernel=False, after=None):
        ctx.profile(per_kernel)
        ms = []
        prev = None
        for i in range(k):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = fn()
            if after is not None:
                after()
            b.record(stream)
            if prev is not None:  # the previous step: wait for its end (this step is queued behind it)
                prev[2].synchronize()
                release(prev[0])
                ms.append(prev[1].elapsed_time(prev[2]))
            prev = (r, a, b)
        barrier()
        prev[2].synchronize()
        release(prev[0])
        ms.append(prev[1].elapsed_time(prev[2]))
        prof = ctx.profile_read() if per_kernel else {}
        ctx.profile(False)
        return ms, prof

    step_ms, _ = timed_steps(lambda: step(src_d, dst_d), args.steps)
    # ---- kernel timing pass: the same steps again, every library kernel
    # bracketed by CUDA events on the stream it is launched on (per-kernel
    # events launch the sequence directly instead of as a graph)
    prof, prof_step_ms = {}, []
    if not args.no_kernel_timing:
        prof_step_ms, prof = timed_steps(lambda: step(src_d, dst_d), args.steps, per_kernel=True)
    clk = clocks.stop()
    t_ms = max_over_ranks(sum(step_ms))
    job_total = replicas.sum_over_ranks(total, dist, "cuda")  # packets of one step, all ranks
    value = replicas.job_rate(job_total * args.steps, t_ms / 1e3)

    # ---- roofline: the whole path (bytes the method must move), and the dominant kernel
    peak, peak_kind = hbm_peak()
    path_gbs = alg_bytes * args.steps / (t_ms / 1e3) / 1e9
    fp = library_fingerprint()
    traffic = None
    rec = NCU_TRAFFIC.get(cfg)
    if not (rec and rec["library"] == fp and rec["matrices"] == with_mats and tuning
            and all(tuning.get(k) == v for k, v in rec["paths"].items())):
        rec = None
    if rec:
        traffic = int(rec["step"] * total)
    roof = {"bound": "hbm", "achieved": round(path_gbs, 1), "peak": peak, "unit": "GB/s",
            "frac": round(path_gbs / peak, 5), "traffic": traffic, "scope": "whole step (every kernel)",
            "bytes_per_step": alg_bytes, "ms_per_step": round(t_ms / args.steps, 4),
            "bytes_rule": "8 B per packet + 72 B per window" + (" + 12 B per window link and row + 8" if with_mats
                                                               else "") + " + 12 B per summed link and row + 80",
            "peak_kind": f"of {peak_kind}", "library": fp}
    dom = max(prof.items(), key=lambda kv: kv[1][1]) if prof else None
    launches = sum(n for n, _ in prof.values())
    kroof = None
    if dom is not None:
        name, (n_l, ms_l) = dom
        mean_ms = ms_l / n_l
        per_step = kernel_bytes_per_step(name, sizes, quants, sum_q, tuning, with_mats)
        if per_step is not None:
            per_launch = int(per_step / (n_l / args.steps))
            ach = per_launch / (mean_ms / 1e3) / 1e9
            kt = rec["kernels"].get(name) if rec else None
            kroof = {"kernel": name, "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(ach / peak, 4), "mean_launch_ms": round(mean_ms, 5),
                     "traffic": int(kt * total) if kt else None,
                     "bytes_per_launch": per_launch, "peak_kind": f"of {peak_kind}",
                     "bytes_rule": "reads + writes each item needs once per launch of this kernel"}
    kernel_share = {k: round(v[1] / max(sum(x[1] for x in prof.values()), 1e-9), 4) for k, v in prof.items()}

    # ---- optional comparator: a library radix sort of the same packed keys
    # (torch.sort on int64, stable: CUB's radix sort of keys with int64
    # indices), against the path's own packet sort (eight passes carrying
    # 16-bit window ids)
    lib_sort = None
    if args.library_sort:
        keys = (src_d.to(torch.int64) & 0xFFFFFFFF) << 32 | (dst_d.to(torch.int64) & 0xFFFFFFFF)
        keys ^= -(1 << 63)  # unsigned order of src << 32 | dst as signed int64 order
        for _ in range(2):
            torch.sort(keys, stable=True)
        torch.cuda.synchronize()
        ls_ms = []
        for i in range(max(1, min(args.steps, 5))):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            torch.sort(keys, stable=True)
            b.record(stream)
            b.synchronize()
            ls_ms.append(a.elapsed_time(b))
        del keys
        torch.cuda.empty_cache()
        own = prof.get("onesweep_pk") or prof.get("onesweep")
        lib_sort = {"what": "torch.sort(stable=True) of the step's packets as int64 keys (CUB radix sort, "
                            "keys + int64 indices)", "ms": round(min(ls_ms), 3),
                    "own_sort_ms": round(own[1] / args.steps, 3) if own else None,
                    "own_sort": "the path's eight digit passes per step (onesweep_pk or onesweep)"}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        src_e = torch.empty_like(src_d)
        dst_e = torch.empty_like(dst_d)

        def e2e_step():
            src_e.copy_(src_h, non_blocking=True)
            dst_e.copy_(dst_h, non_blocking=True)
            return step(src_e, dst_e)

        def d2h():
            q_host.copy_(q_dev, non_blocking=True)

        for _ in range(2):
            r = e2e_step()
            d2h()
            torch.cuda.synchronize()
            release(r)
        barrier()
        e2e_ms, _ = timed_steps(e2e_step, args.steps, after=d2h)
        e2e_t = max_over_ranks(sum(e2e_ms))
        staged = {"value": replicas.job_rate(job_total * args.steps, e2e_t / 1e3), "unit": UNIT,
                  "h2d_bytes_per_step": 8 * total, "d2h_bytes_per_step": 72 * nwin,
                  "how": "cudaMemcpyAsync of the pairs from pinned host memory into device buffers, then "
                         "ans_batch_submit_host"}

        # Pipelined: step i+1's pairs are copied (a second stream, two device
        # buffers) while step i is analysed; every step still copies its
        # pairs in and its quantities out inside the timed region.
        def pipelined(k):
            copy = torch.cuda.Stream()
            bufs = ((src_d, dst_d), (src_e, dst_e))
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            done = []
            t0.record(stream)
            copy.wait_event(t0)
            prev = None
            for i in range(k):
                s_b, d_b = bufs[i % 2]
                if i >= 2:
                    copy.wait_event(done[i - 2])  # the batch that last read this buffer
                with torch.cuda.stream(copy):
                    s_b.copy_(src_h, non_blocking=True)
                    d_b.copy_(dst_h, non_blocking=True)
                    copied = torch.cuda.Event()
                    copied.record(copy)
                flush.fill_(i & 0xFF)
                stream.wait_event(copied)
                r = step(s_b, d_b)
                d2h()
                ev = torch.cuda.Event()
                ev.record(stream)
                done.append(ev)
                if prev is not None:  # keep at most two steps' results alive
                    done[i - 1].synchronize()
                    release(prev)
                prev = r
            t1.record(stream)
            t1.synchronize()
            release(prev)
            return t0.elapsed_time(t1)

        pipelined(2)
        barrier()
        pl_t = max_over_ranks(pipelined(args.steps))
        pipe = {"value": replicas.job_rate(job_total * args.steps, pl_t / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": 8 * total, "d2h_bytes_per_step": 72 * nwin,
                "how": "as staged, with step i+1's copies (second stream, two device buffers) overlapping the "
                       "analysis of step i; K steps between CUDA events"}
        del src_e, dst_e

        # The same call given the pinned host arrays themselves: the batch's
        # kernels read the pairs in place over the host link (the packet pack
        # reads each pair once), so the transfer happens inside the batch.
        def ip_step():
            return step(src_h, dst_h)

        for _ in range(2):
            r = ip_step()
            d2h()
            torch.cuda.synchronize()
            release(r)
        barrier()
        ip_ms, _ = timed_steps(ip_step, args.steps, after=d2h)
        ip_t = max_over_ranks(sum(ip_ms))
        in_place = {"value": replicas.job_rate(job_total * args.steps, ip_t / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": 8 * total, "d2h_bytes_per_step": 72 * nwin,
                    "how": "ans_batch_submit_host given the pinned host arrays: the kernels read the pairs in place"}
        # the headline: the fastest of the three ways of feeding host-resident
        # pairs (pipelining pays off on large batches, reading in place on small ones)
        ways = {"pipelined": pipe, "in_place": in_place, "staged": staged}
        best = max(ways, key=lambda k: ways[k]["value"])
        e2e = {"value": ways[best]["value"], "unit": UNIT, "h2d_bytes_per_step": 8 * total,
               "d2h_bytes_per_step": 72 * nwin, "path": best, **ways}

        # The same through ans_batch_submit_windows: the batch kernels read
        # every window's pairs in place from the pinned host arrays (the
        # host-to-device transfer happens inside the timed kernels).
        wins = [(src_h[int(a):int(b)], dst_h[int(a):int(b)]) for a, b in zip(w.offsets[:-1], w.offsets[1:])]

        def zc_step():
            mats, summ, _ = ctx.batch_submit_windows(wins, flags, out=q_dev, want_ticket=False)
            return mats, summ

        for _ in range(2):
            r = zc_step()
            d2h()
            torch.cuda.synchronize()
            release(r)
        barrier()
        zc_ms, _ = timed_steps(zc_step, args.steps, after=d2h)
        zc_t = max_over_ranks(sum(zc_ms))
        e2e["zero_copy"] = {"value": replicas.job_rate(job_total * args.steps, zc_t / 1e3), "unit": UNIT,
                            "h2d_bytes_per_step": 8 * total, "d2h_bytes_per_step": 72 * nwin,
                            "how": "ans_batch_submit_windows: the kernels read each window's pairs in place "
                                   "from pinned host memory"}

    # ---- the plain per-window method on the same GPU
    per_window = None
    if not args.no_per_window:
        k2 = max(1, min(args.steps, 3))

        def pw_step():
            mats = []
            for i in range(nwin):
                a, b = int(w.offsets[i]), int(w.offsets[i + 1])
                mats.append(ctx.build_window(src_d[a:], dst_d[a:], b - a))
            return mats, ctx.sum_windows(mats)

        release(pw_step())
        torch.cuda.synchronize()
        barrier()
        pw_ms, _ = timed_steps(pw_step, k2)
        pw_t = max_over_ranks(sum(pw_ms))
        per_window = {"value": replicas.job_rate(job_total * k2, pw_t / 1e3), "unit": UNIT, "steps": k2,
                      "ms_per_step": pw_t / k2, "launches": f"{nwin} x ans_build_window + ans_sum_windows"}
    ctx.close()
    del src_d, dst_d, flush

    # ---- CPU oracle baseline (rank 0, N=1 only): all cores and one core
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores, model = host_cpu()
        ns = max(1, min(nwin, ORACLE_SAMPLE[cfg]))
        sample = w.subset(0, ns)
        pool = OraclePool(sample, cores)
        try:
            pk, dt = pool.run()
        finally:
            pool.close()
        v1, n1, dt1 = time_oracle_one_core(w)
        cpu = {"value": pk / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu_model": model,
               "sample": f"first {ns} of {nwin} windows ({pk} packets) + their time sum, {dt:.1f} s; numpy "
                         f"oracle, a process per core over windows, the ranges' sums added",
               "one_core": {"value": v1, "unit": UNIT, "cores": 1,
                            "sample": f"first {n1} of {nwin} windows + their time sum ({dt1:.1f} s)"}}

    serving = None
    if rank == 0 and not args.no_serve:
        from paper_2510_14050_gb300 import serve
        spool = serve.pool_source(512, seed=0)
        stun = None if args.serve_no_autotune else serving_tuning(local, spool)
        serving, _ = run_serving(local, args.serve_rate, args.serve_windows, args.serve_budget_gib, spool,
                                 tuning=stun, batch_windows=args.serve_batch_windows,
                                 batch_packets=args.serve_batch_packets)

    # ---- out of core: the step's windows streamed from pinned host memory
    out_of_core = None
    if args.stream_batches > 0:
        from paper_2510_14050_gb300 import stream
        bp = int(-(-total // args.stream_batches))
        stream.stream_windows(src_h, dst_h, w.offsets, batch_packets=bp, tuning=tuning).sum.free()  # warm-up
        res = stream.stream_windows(src_h, dst_h, w.offsets, batch_packets=bp, tuning=tuning)
        res.sum.free()
        s_max = max_over_ranks(res.seconds)
        out_of_core = {"value": replicas.job_rate(job_total, s_max), "unit": UNIT, "batches": res.batches,
                       "batch_packets": bp, "seconds": s_max,
                       "over_staged_e2e": (replicas.job_rate(job_total, s_max) / e2e["staged"]["value"]) if e2e
                       else None,
                       "timeline_ms": res.timeline,
                       "what": "windows streamed from pinned host memory, two batches in flight "
                               "(H2D of one overlapped with the analysis of the other); time sum folded on the "
                               "device; timeline = per batch (slot, H2D start, H2D end, analysis end) in ms"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "ms_per_step_min": round(min(step_ms), 4), "ms_per_step_median": round(statistics.median(step_ms), 4),
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOADS[cfg], "config": cfg, "windows": nwin, "packets_per_step": total,
                       "per_window_matrices": with_mats,
                       "l2": "flushed between timed steps (512 MiB write)", "parallelism": f"replicas x{world}"},
            "e2e": e2e, "gpu_launches": launches, "roofline": roof, "kernel_roofline": kroof,
            "per_window": per_window,
            "batched_over_per_window": (value / per_window["value"]) if per_window else None,
            "kernel_time_share": kernel_share,
            "kernel_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in prof.items()},
            "kernel_timing": {"how": "a second pass of the same steps with CUDA events around every library "
                                     "kernel on its launching stream (launched directly, not as a graph)",
                              "ms_per_step": round(max_over_ranks(sum(prof_step_ms)) / args.steps, 4)
                              if prof_step_ms else None},
            "time_sum": {"unique_links": sum_q["unique_links"], "unique_sources": sum_q["unique_sources"],
                         "unique_destinations": sum_q["unique_destinations"],
                         "window_links": sum(q["unique_links"] for q in quants)},
            "tuning": tuning, "serving": serving, "out_of_core": out_of_core, "clocks": clk, "cpu_baseline": cpu,
            "library_sort": lib_sort,
            "setup_s": {"generate": round(t_gen, 2), "autotune": round(t_tune, 2)},
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
