#!/usr/bin/env python3
"""Throughput of the batched anonymized-network-sensing path on GB300.

One step = one pass of the whole hot path over one batch of synthetic
windows: pack + sort + run-length reduction to per-window DCSR matrices, the
nine quantities of every window, and the time sum of all windows of the batch
(its DCSR and quantities).  The default workload is the 64-window batch
(64 x 2^17 packets, src Zipf(1.1)/2^20, dst Zipf(1.3)/2^22, 5% bursts).

Prints ONE JSON line (rank 0).  Fields beyond the base contract:
  per_window   the same work as 64 separate ans_build_window calls + one
               ans_sum_windows (the plain one-window-per-launch method)
  roofline     dominant kernel: algorithmic bytes per launch / mean launch
               time against the measured HBM copy bandwidth.  The timed
               region runs the production path (every batch replayed as a
               CUDA graph); the launch times come from a second timed pass
               over the same steps with CUDA events around every library
               kernel on its launching stream (kernel_timing)
  path_roofline  the whole step's algorithmic bytes / step time
  cpu_baseline the CPU oracle timed on this host on a bounded sample

`--impl reference` times the CPU oracle instead (the reference arm).
Multi-GPU (torchrun): independent replicas, one batch of distinct windows per
rank, barrier + max-over-ranks timing, weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "packets/s (batched hot path: per-window DCSR + 9 quantities + time sum)"
UNIT = "packets/s"
FLUSH_BYTES = 512 << 20  # > 129 MB L2
FALLBACK_HBM_GBS = 6800.0

WORKLOADS = {
    1: "1 window x 2^17 packets; src, dst Zipf(1.2)/2^16; DCSR + 9 quantities (the plain single-window case)",
    2: "64 windows x 2^17 packets (8.4M pairs); src Zipf(1.1)/2^20, dst Zipf(1.3)/2^22, 5% bursts of 2..100; "
       "per-window DCSR + 9 quantities + 64-window time sum",
    3: "1024 windows, P loguniform [2^10, 2^20]; heavy hitter 10%, scanners, rest Zipf(1.1)/2^24; "
       "per-window DCSR + 9 quantities + time sum",
    4: "2^13 windows x 2^17 (2^30 pairs); src, dst Zipf(1.05) over 2^32; per-window DCSR + quantities + time sum",
}
DEFAULT_NWIN = {1: 1, 2: 64, 3: 1024, 4: 8192}

# ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_onesweep launch
# (64-bit link keys, first digit pass) on the 64-window batch, cold cache; set
# to None whenever that kernel changes until it is captured again.
ONESWEEP_NCU_TRAFFIC = 92343552  # 69165056 + 23178496 B, pass 0, cold cache


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", type=int, default=2, choices=sorted(WORKLOADS))
    ap.add_argument("--nwin", type=int, default=None, help="override the number of windows per step")
    ap.add_argument("--impl", default="ans", choices=["ans", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-per-window", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tuning", default=None,
                    help="fix launch shapes and paths instead of autotuning, e.g. key=512,0,2;kv=512,0,1;agg_path=1")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--stream-batches", type=int, default=4,
                    help="out-of-core run: the step's windows streamed from pinned host memory in this many "
                         "batches, two in flight (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=1e4, help="serving arrivals, windows/s")
    ap.add_argument("--serve-windows", type=int, default=20000)
    ap.add_argument("--serve-budget-gib", type=float, default=64.0)
    ap.add_argument("--serve-sweep", action="store_true",
                    help="only serving: every rate of 1e3..1e5 windows/s x budgets 32/64/128 GiB, one line each")
    return ap.parse_args()


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


def algorithmic_bytes(sizes, quants, sum_q):
    """Sec. 8(d) bytes of one step: read pairs, write DCSR + quantities per
    window, write the time-summed DCSR + quantities."""
    b = 0
    for p, q in zip(sizes, quants):
        b += 8 * int(p) + 12 * q["unique_links"] + 12 * q["unique_sources"] + 8 + 72
    if sum_q is not None:
        b += 12 * sum_q["unique_links"] + 12 * sum_q["unique_sources"] + 8 + 72
    return b


def kernel_bytes_per_step(name, sizes, quants, sum_q, tuning):
    """Algorithmic bytes one step's launches of kernel family `name` move
    (reads + writes each item needs once per pass; DESIGN lists the rules).
    P = packets (split by window-sort path), U/R = links/rows of the windows,
    Us/Rs = links/rows of the time sum."""
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
    rules = {
        "pack_hist": 16 * p_os,                        # read pairs, write keys
        "onesweep": 8 * 16 * p_os,                     # 8 passes: read + write a key
        "cluster_sort": 16 * p_cl,                     # read pairs, write sorted keys
        "hash_insert": 8 * p_all,                      # read pairs
        "hash_compact": 32 * u,                        # slot in, (key, count) out
        "onesweep_hash": 8 * 32 * u,                   # 8 passes over (key, count)
        "rle": 8 * p_all + 12 * u + 20 * r + 8 * u + 12 * us + 20 * rs,
        "finish": 32 * u + 32 * r + 28 * us + 32 * rs,
        "onesweep_col": 4 * 16 * u + 4 * 24 * us,      # (dst, u32 count) / (dst, u64 count)
        "colstat": 8 * u + 12 * us,
        "gather": 28 * u,                              # link + its row in, (key, count) out
        "merge": rounds * 32 * u,                      # each round: read both runs, write the merge
        "onesweep_sum": 8 * 32 * u,                    # 8 passes over (key, count)
        "scan_u64": 16 * u,
    }
    return rules.get(name)


def run_serving(local, rate, n, budget_gib, pool=None, seed=0):
    """Open-loop Poisson arrivals of serving-size windows (P uniform in
    [2^12, 2^17], traffic as the 64-window batch) through the
    continuous-batching server; latency from arrival to quantities on the host,
    H2D included.  Running 1-minute and 1-hour tumbling sums stay resident."""
    from paper_2510_14050_gb300 import serve
    pool = pool or serve.pool_source(512, seed=seed)
    npool = pool.offsets.size - 1
    srv = serve.Server(device=local, slots=4, budget_bytes=int(budget_gib * (1 << 30)), max_batch_windows=256,
                       max_batch_packets=1 << 24, bucket_seconds=(60.0, 3600.0))
    try:
        warm_t, warm_o = serve.poisson_schedule(rate, min(n, 200), npool, seed=seed + 1)
        srv.serve(pool, warm_t, warm_o)
        arr, order = serve.poisson_schedule(rate, n, npool, seed=seed)
        st = srv.serve(pool, arr, order)
        out = {"lambda_windows_per_s": rate, "budget_gib": budget_gib, "slots": 4, **st.summary(),
               "offered_packets_per_s": float(np.diff(pool.offsets)[order].sum() / max(arr[-1], 1e-9))}
    finally:
        srv.close()
    return out, pool


def oracle_step(w):
    import oracle
    oracle.batch(w.src, w.dst, w.offsets, want_sum=True)


def time_oracle(w, budget_s=12.0):
    """Run the oracle over windows of `w` until ~budget_s has elapsed (at
    least one window); return (packets/s, windows used)."""
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
    sample = max(1, min(nwin, 8))
    w = synth.generate(args.config, nwin=sample)
    for _ in range(args.warmup):
        oracle_step(w.subset(0, 1))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_step(w)
    dt = time.perf_counter() - t0
    value = w.total * args.steps / dt
    sample_desc = f"first {sample} of {nwin} windows ({w.total} packets) + their time sum, per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.config], "sample": sample_desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample_desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch

    from paper_2510_14050_gb300 import ans, replicas, synth

    torch.cuda.set_device(local)
    if args.serve_sweep:
        if rank == 0:
            pool = None
            for budget in (32.0, 64.0, 128.0):
                for rate in (1e3, 3e3, 1e4, 3e4, 1e5):
                    n = max(args.serve_windows, int(min(rate * 10.0, 200000)))
                    res, pool = run_serving(local, rate, n, budget, pool)
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
    w = synth.generate(cfg, nwin=nwin, first_window=replicas.first_window(rank, nwin))
    total = w.total
    sizes = np.diff(w.offsets)

    ctx = ans.Context(local)
    stream = torch.cuda.current_stream()
    tuning = None
    src_h = torch.from_numpy(w.src.view(np.int32)).pin_memory()
    dst_h = torch.from_numpy(w.dst.view(np.int32)).pin_memory()
    src_d = src_h.cuda()
    dst_d = dst_h.cuda()
    q_dev = torch.zeros((nwin, 9), dtype=torch.int64, device="cuda")
    q_host = torch.zeros((nwin, 9), dtype=torch.int64).pin_memory()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    flags = ans.BATCH_MATRICES | ans.BATCH_SUM

    def step(s, d):
        mats, summ, _ = ctx.batch_submit(s, d, w.offsets, flags, out=q_dev, want_ticket=False)
        return mats, summ

    def release(res):
        mats, summ = res
        for m in mats:
            m.free()
        summ.free()

    if args.tuning:
        kw = {}
        for part in args.tuning.split(";"):
            fam, vals = part.split("=")
            fam = fam.strip()
            if fam.endswith("_path") or fam in ("col_hash", "merge_tile"):  # e.g. agg_path=1; graph_path=0 sets graph
                kw["graph" if fam == "graph_path" else fam] = int(vals)
                continue
            for field, v in zip(("threads", "rank", "blocks"), vals.split(",")):
                kw[f"{fam}_{field}"] = int(v)
        ctx.set_tuning(**kw)
        tuning = ctx.get_tuning()
    elif not args.no_autotune:
        tuning = ctx.autotune(src_d, dst_d, w.offsets)
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
    alg_bytes = algorithmic_bytes(sizes, quants, sum_q)

    # ---- timed region: device-resident inputs, the production path (each
    # batch's launch sequence replayed as a CUDA graph), no per-kernel events
    clocks = ClockSampler(local)
    barrier()
    clocks.start()

    def timed_steps(per_kernel: bool):
        ctx.profile(per_kernel)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        keep = []
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            evs[i][0].record(stream)
            keep.append(step(src_d, dst_d))
            evs[i][1].record(stream)
        barrier()
        prof = ctx.profile_read() if per_kernel else {}
        ctx.profile(False)
        ms = [a.elapsed_time(b) for a, b in evs]
        for r in keep:
            release(r)
        return ms, prof

    step_ms, _ = timed_steps(False)
    # ---- kernel timing pass: the same steps again, every library kernel
    # bracketed by CUDA events on the stream it is launched on (per-kernel
    # events launch the sequence directly instead of as a graph)
    prof_step_ms, prof = timed_steps(True)
    clk = clocks.stop()
    t_ms = max_over_ranks(sum(step_ms))
    job_total = replicas.sum_over_ranks(total, dist, "cuda")  # packets of one step, all ranks
    value = replicas.job_rate(job_total * args.steps, t_ms / 1e3)

    # ---- dominant kernel and roofline
    peak, peak_kind = hbm_peak()
    dom = max(prof.items(), key=lambda kv: kv[1][1]) if prof else None
    launches = sum(n for n, _ in prof.values())
    roof = None
    if dom is not None:
        name, (n_l, ms_l) = dom
        mean_ms = ms_l / n_l
        per_step = kernel_bytes_per_step(name, sizes, quants, sum_q, tuning)
        per_launch = int(per_step / (n_l / args.steps)) if per_step is not None else alg_bytes
        unit_desc = {"onesweep": "16 B per packet per digit pass",
                     "merge": "32 B per window link per merge round",
                     "onesweep_sum": "32 B per window link per digit pass",
                     "onesweep_col": "16 B per window link (u32 count) / 24 B per time-sum link per digit pass",
                     "cluster_sort": "16 B per packet"}.get(name, "per-kernel algorithmic bytes" if per_step
                                                            else "whole-step algorithmic bytes")
        ach = per_launch / (mean_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "traffic": ONESWEEP_NCU_TRAFFIC if name == "onesweep" else None,
                "kernel": name, "mean_launch_ms": round(mean_ms, 5), "bytes_per_launch": per_launch,
                "bytes_rule": unit_desc, "peak_kind": f"of {peak_kind}"}
    path_gbs = alg_bytes * args.steps / (t_ms / 1e3) / 1e9
    kernel_share = {k: round(v[1] / max(sum(x[1] for x in prof.values()), 1e-9), 4) for k, v in prof.items()}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        src_e = torch.empty_like(src_d)
        dst_e = torch.empty_like(dst_d)
        for _ in range(2):
            src_e.copy_(src_h, non_blocking=True)
            dst_e.copy_(dst_h, non_blocking=True)
            r = step(src_e, dst_e)
            q_host.copy_(q_dev, non_blocking=True)
            torch.cuda.synchronize()
            release(r)
        barrier()
        evs2 = []
        keep = []
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            src_e.copy_(src_h, non_blocking=True)
            dst_e.copy_(dst_h, non_blocking=True)
            keep.append(step(src_e, dst_e))
            q_host.copy_(q_dev, non_blocking=True)
            b.record(stream)
            evs2.append((a, b))
        barrier()
        e2e_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs2))
        for r in keep:
            release(r)
        e2e = {"value": replicas.job_rate(job_total * args.steps, e2e_ms / 1e3), "unit": UNIT,
               "h2d_bytes_per_step": 8 * total, "d2h_bytes_per_step": 72 * nwin}

        # The same through ans_batch_submit_windows: the batch kernels read
        # every window's pairs in place from the pinned host arrays (the
        # host-to-device transfer happens inside the timed kernels).
        wins = [(src_h[int(a):int(b)], dst_h[int(a):int(b)]) for a, b in zip(w.offsets[:-1], w.offsets[1:])]

        def zc_step():
            mats, summ, _ = ctx.batch_submit_windows(wins, flags, out=q_dev, want_ticket=False)
            return mats, summ

        for _ in range(2):
            r = zc_step()
            q_host.copy_(q_dev, non_blocking=True)
            torch.cuda.synchronize()
            release(r)
        barrier()
        evs4, keep = [], []
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            keep.append(zc_step())
            q_host.copy_(q_dev, non_blocking=True)
            b.record(stream)
            evs4.append((a, b))
        barrier()
        zc_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs4))
        for r in keep:
            release(r)
        e2e["zero_copy"] = {"value": replicas.job_rate(job_total * args.steps, zc_ms / 1e3), "unit": UNIT,
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
        evs3, keep = [], []
        for i in range(k2):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            keep.append(pw_step())
            b.record(stream)
            evs3.append((a, b))
        barrier()
        pw_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs3))
        for r in keep:
            release(r)
        per_window = {"value": replicas.job_rate(job_total * k2, pw_ms / 1e3), "unit": UNIT, "steps": k2,
                      "ms_per_step": pw_ms / k2, "launches": f"{nwin} x ans_build_window + ans_sum_windows"}

    # ---- CPU oracle baseline (rank 0, N=1 only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, n_used, dt = time_oracle(w)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {n_used} of {nwin} windows + their time sum ({dt:.1f} s, numpy, 1 thread)"}

    serving = None
    if rank == 0 and not args.no_serve:
        serving, _ = run_serving(local, args.serve_rate, args.serve_windows, args.serve_budget_gib)

    # ---- out of core: the step's windows streamed from pinned host memory
    out_of_core = None
    if args.stream_batches > 0:
        from paper_2510_14050_gb300 import stream
        bp = int(-(-total // args.stream_batches))
        stream.stream_windows(src_h, dst_h, w.offsets, batch_packets=bp).sum.free()  # warm-up
        res = stream.stream_windows(src_h, dst_h, w.offsets, batch_packets=bp)
        res.sum.free()
        s_max = max_over_ranks(res.seconds)
        out_of_core = {"value": replicas.job_rate(job_total, s_max), "unit": UNIT, "batches": res.batches,
                       "batch_packets": bp, "seconds": s_max,
                       "what": "windows streamed from pinned host memory, two batches in flight "
                               "(H2D of one overlapped with the analysis of the other); time sum folded on the device"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": WORKLOADS[cfg], "windows": nwin, "packets_per_step": total,
                       "l2": "flushed between timed steps (512 MiB write)", "parallelism": f"replicas x{world}"},
            "e2e": e2e, "gpu_launches": launches, "roofline": roof,
            "path_roofline": {"achieved": round(path_gbs, 1), "peak": peak, "unit": "GB/s",
                              "frac": round(path_gbs / peak, 4), "bytes_per_step": alg_bytes},
            "per_window": per_window,
            "batched_over_per_window": (value / per_window["value"]) if per_window else None,
            "kernel_time_share": kernel_share,
            "kernel_ms_per_step": {k: round(v[1] / args.steps, 4) for k, v in prof.items()},
            "kernel_timing": {"how": "a second pass of the same steps with CUDA events around every library "
                                     "kernel on its launching stream (launched directly, not as a graph)",
                              "ms_per_step": round(max_over_ranks(sum(prof_step_ms)) / args.steps, 4)},
            "tuning": tuning, "serving": serving, "out_of_core": out_of_core, "clocks": clk, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
