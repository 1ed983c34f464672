#!/usr/bin/env python3
"""Benchmark: kNN (k=20) + regularised covariance of a 131k-point ray-cast
LiDAR scan against a 2M-point race-track map, on one GB300 per rank.

A step is one pass of the whole path over one scan: pc_knn_cov (search +
covariance + plane regularisation) with the map grid resident.  The timed
value is device time (CUDA events on the launching stream) with inputs in
HBM and L2 flushed (a 256 MB write) before every timed step, outside the
events.  `e2e` repeats the step through the host-buffer entry
pc_knn_cov_host with page-locked host buffers (the search reads the scan
and writes idx/d2/cov in host memory itself), every host<->device transfer
inside the timed region.

Multi-GPU (torchrun): every rank processes its own scan per step against
its own copy of the map -- queries shard with no data-path collective
(weak scaling); only the barrier and the max-over-ranks timing use
torch.distributed.

--impl reference times the CPU oracle (k-d tree kNN + binary64 covariance,
tree build excluded) on the host cores, on a bounded sample of the same
scan per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "query points/sec for kNN(k=20)+cov, 131k scan vs 2M map; p99 scan latency; % HBM peak"
UNIT = "points/s"
K_NN = 20
EPS = 1e-3
MAP_POINTS = 2_000_000
FLUSH_BYTES = 256 << 20  # > 129 MB L2
FALLBACK_HBM_GBS = 6800.0
TIMED_DEVICE_MS = 1200.0  # device time the C2 timed region aims for
SEARCH_KERNEL = "k_knn<0,1,0> (fused search + covariance, whole-map variant)"
KERNEL_SOURCES = ["paper_2308_07173_gb300/csrc/knn_kernels.cuh", "paper_2308_07173_gb300/csrc/pc_device.cuh",
                  "paper_2308_07173_gb300/csrc/pc_search.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "knn_cov_c2_ncu.json")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def measured_profile():
    """The committed ncu capture of the search kernel (dram bytes and warp
    instructions per launch), valid only while the kernel source is
    unchanged; None otherwise."""
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
        if d.get("source_sha") != kernel_source_hash():
            return None
        return d
    except Exception:
        return None


def measured_traffic():
    """dram bytes per launch of the search kernel (committed capture)."""
    d = measured_profile()
    try:
        return float(d["dram_bytes_per_launch_full_size"]) if d else None
    except (KeyError, TypeError, ValueError):
        return None


def l2_figures(ms_per_launch):
    """L2 traffic of the search kernel from the committed capture (lts__t_bytes
    per launch, valid while the kernel source is unchanged) over the measured
    launch time, beside its DRAM bytes."""
    d = measured_profile()
    if not d or "l2_bytes_per_launch" not in d:
        return None
    l2b = float(d["l2_bytes_per_launch"])
    out = {"l2_bytes_per_launch": l2b, "achieved_l2_gbs": l2b / (ms_per_launch / 1e3) / 1e9,
           "dram_bytes_per_launch": d.get("dram_bytes_per_launch_full_size"),
           "source": "lts__t_bytes.sum and dram__bytes of the committed ncu capture "
                     "(profiles/knn_cov_c2_ncu.json), over this run's launch time"}
    if "candidates_per_query" in d:
        out["candidates_per_query"] = d["candidates_per_query"]
        out["candidate_bytes_per_launch"] = d.get("candidate_bytes_per_launch")
    return out


def issue_roofline(ms_per_launch, clk, sms):
    """Instruction-issue roofline of the search kernel: its warp
    instructions per launch (committed capture) over the measured launch
    time, against 4 warp instructions per cycle per SM (one issue slot per
    sub-partition) at the median SM clock sampled during the timed region."""
    d = measured_profile()
    try:
        inst = float(d["warp_instructions_per_launch"]) if d else None
    except (KeyError, TypeError, ValueError):
        inst = None
    mhz = (clk or {}).get("sm_mhz") or (clk or {}).get("sm_max_mhz")
    if inst is None or not mhz or not sms:
        return None
    achieved = inst / (ms_per_launch / 1e3) / 1e12
    peak = 4.0 * sms * mhz * 1e6 / 1e12
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "Twarp-inst/s",
            "frac": achieved / peak, "warp_instructions_per_launch": inst, "sm_count": sms, "sm_mhz": mhz,
            "source": "smsp__inst_executed.sum of the committed ncu capture (profiles/knn_cov_c2_ncu.json)"}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 50):
        self.idx = gpu_index
        self.interval = int(interval_ms)
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.interval), "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
            os.unlink(self.path)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    from paper_2308_07173_gb300 import workloads as W

    q, m = W.scan_vs_map(MAP_POINTS)
    oracle.build()
    tree = oracle.KDTree(m)
    threads = oracle.default_threads()
    # bounded sample per step: a contiguous slice of the scan, sized so each
    # step is ~1-3 s on the host
    S = min(len(q), args.ref_sample)
    times = []
    for step in range(args.warmup + args.steps):
        lo = (step * S) % max(1, len(q) - S)
        qs = q[lo:lo + S]
        t0 = time.perf_counter()
        idx, _ = tree.knn(qs, K_NN, threads=threads)
        oracle.cov(m, idx, EPS, threads=threads)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = S * len(times) / total
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": "c2_scan131k_vs_map2M_k20_eps1e-3", "n_queries_per_step": S, "k": K_NN,
                   "eps": EPS, "map_points": MAP_POINTS},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{S} consecutive queries of the 131k scan per step; k-d tree kNN + binary64 covariance; tree build excluded"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(q, m, budget_s: float = 20.0):
    import numpy as np

    import oracle

    oracle.build()
    threads = oracle.default_threads()
    t0 = time.perf_counter()
    tree = oracle.KDTree(m)
    build_s = time.perf_counter() - t0
    # grow the sample until it takes a few seconds, within the budget
    S = 4096
    while True:
        qs = q[:S]
        t0 = time.perf_counter()
        idx, _ = tree.knn(qs, K_NN, threads=threads)
        oracle.cov(m, idx, EPS, threads=threads)
        dt = time.perf_counter() - t0
        if dt > 2.0 or S >= len(q) or dt * (2 * S / S) > budget_s:
            break
        S = min(len(q), S * 4)
    return {"value": S / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {S} queries of the 131k scan; k-d tree kNN (k=20) + binary64 covariance with "
                      f"plane regularisation; tree build ({build_s:.1f} s) excluded"}


# ---------------------------------------------------------------- GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--ref-sample", type=int, default=16384)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4", "c5", "gicp", "window", "kernel", "wall", "append"],
                    help="c2 is the headline; the others print their own line")
    ap.add_argument("--duration", type=float, default=10.0, help="c4: seconds of arrivals")
    ap.add_argument("--lambdas", default="0.5,1,2,4", help="c4: arrival-rate multiples swept")
    ap.add_argument("--served-duration", type=float, default=2.0,
                    help="seconds of arrivals in the C2 line's served sub-object")
    ap.add_argument("--scans-per-step", type=int, default=0,
                    help="c2: scans per timed step (0: enough for about a second of device time)")
    ap.add_argument("--headline-only", action="store_true",
                    help="c2: skip the batched and served sub-objects")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "c2":
        return {"c1": run_c1, "c3": run_c3, "c4": run_c4, "c5": run_c5, "gicp": run_gicp,
                "window": run_window, "kernel": run_kernel, "wall": run_wall,
                "append": run_append}[args.workload](args)
    return run_c2(args)


def algorithmic_roofline(md, info, idx_list, n_queries: int, k: int, ms: float) -> dict:
    """HBM roofline of one search launch: algorithmic bytes N (12 + 8k + 24)
    + 12 U_p + 8 U_c (U_p distinct target points in the answers, U_c the
    distinct cells holding them) over the launch time, against the measured
    copy bandwidth."""
    import torch

    ui = torch.unique(torch.cat([i.reshape(-1) for i in idx_list]).long())
    ui = ui[ui >= 0]
    U_p = int(ui.numel())
    pts = md[ui]
    o = torch.tensor(info["origin"], device=md.device)
    cells = torch.floor((pts - o) * (1.0 / info["cell_size"])).long()
    ckey = (cells[:, 0] << 42) | (cells[:, 1] << 21) | cells[:, 2]
    U_c = int(torch.unique(ckey).numel())
    alg = n_queries * (12 + 8 * k + 24) + 12 * U_p + 8 * U_c
    peak, kind = peaks()
    achieved = alg / (ms / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": kind, "algorithmic_bytes": alg, "U_p": U_p, "U_c": U_c}


def copy_bandwidth(dev, stream, qh, qd, outs, douts) -> dict:
    """Where the end-to-end time goes: the host-to-device upload of one scan
    and the device-to-host download of its three outputs, each timed alone
    with CUDA events on the bench stream (pinned host buffers, as the host
    entry uses), next to plain device-to-pinned-host copies of 1-64 MB."""
    import torch

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    with torch.cuda.stream(stream):
        up = timed(lambda: qd.copy_(qh, non_blocking=True))
        down = timed(lambda: [h.copy_(d, non_blocking=True) for h, d in zip(outs, douts)])
        out = {"upload_ms": up, "upload_gbs": qh.numel() * 4 / up / 1e6,
               "download_ms": down, "download_gbs": sum(h.numel() * 4 for h in outs) / down / 1e6,
               "d2h_pinned_gbs": {}}
        for mb in (1, 4, 16, 24, 64):
            src = torch.empty(mb << 20, dtype=torch.uint8, device=dev)
            dst = torch.empty(mb << 20, dtype=torch.uint8, pin_memory=True)
            ms = timed(lambda: dst.copy_(src, non_blocking=True))
            out["d2h_pinned_gbs"][f"{mb}MB"] = (mb << 20) / ms / 1e6
    return out


def run_c2(args):
    import torch

    from paper_2308_07173_gb300 import pc, sharding
    from paper_2308_07173_gb300 import workloads as W

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pc.load()

    # rank r answers scan r of the stream (scans_for_rank deals them round-robin)
    (scan_id,) = sharding.scans_for_rank(ws, ws, rank)
    q, m = W.scan_vs_map(MAP_POINTS, scan_seed=3 + scan_id)
    N = len(q)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    md = torch.from_numpy(m).to(dev)
    from paper_2308_07173_gb300 import autotune

    tuned = autotune.lookup(autotune.default_cache(), K_NN, MAP_POINTS, N)
    t = autotune.apply(md, tuned) if tuned else pc.Target(md)
    info = t.info()
    qd = torch.from_numpy(q).to(dev)
    idx = torch.empty((N, K_NN), dtype=torch.int32, device=dev)
    d2 = torch.empty((N, K_NN), dtype=torch.float32, device=dev)
    cov = torch.empty((N, 6), dtype=torch.float32, device=dev)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()

    def scan():
        t.knn_cov(qd, K_NN, EPS, idx, d2, cov, stream=stream)

    warm = []
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            scan()
            b.record(stream)
            warm.append((a, b))
    stream.synchronize()
    assert t.sync_status(stream) == pc.PC_OK
    # A step is R scans back to back, each after an L2 flush, so that the
    # timed region holds about a second of device time whatever --steps is
    # (enough for the clock samples); every scan is timed by its own events.
    est = statistics.median(a.elapsed_time(b) for a, b in warm)
    R = args.scans_per_step or max(1, min(4000, int(math.ceil(TIMED_DEVICE_MS / (args.steps * est)))))
    if dist:
        R = int(sharding.reduce_max(R, dev))
    t.stats(reset=True, stream=stream)

    clocks = Clocks(local)
    clocks.start()
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(R)]
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            for r in range(R):
                flush.fill_(1)
                ev[i][r][0].record(stream)
                scan()
                ev[i][r][1].record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    st = t.sync_status(stream)
    assert st == pc.PC_OK, pc.pc_status_string(st)
    path_stats = t.stats(reset=True, stream=stream)
    scan_ms = [a.elapsed_time(b) for step in ev for a, b in step]
    total_ms = sum(scan_ms)
    total_ms = sharding.reduce_max(total_ms, dev)
    n_all = sharding.reduce_sum(N, dev)
    value = n_all * R * args.steps / (total_ms / 1e3)
    ms_per_step = total_ms / args.steps
    ms_per_scan = total_ms / (args.steps * R)
    lat = sorted(scan_ms)

    roof = algorithmic_roofline(md, info, [idx], N, K_NN, ms_per_scan)
    roof["traffic"] = measured_traffic()
    roof["kernel"] = SEARCH_KERNEL
    l2 = l2_figures(ms_per_scan)

    # end to end through the host-buffer entry
    qh = torch.from_numpy(q).pin_memory()
    outs = (torch.empty((N, K_NN), dtype=torch.int32).pin_memory(),
            torch.empty((N, K_NN), dtype=torch.float32).pin_memory(),
            torch.empty((N, 6), dtype=torch.float32).pin_memory())
    e2e_steps = max(3, min(args.steps, 200))
    e2e_t = []
    for i in range(args.warmup + e2e_steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        stream.synchronize()
        t0 = time.perf_counter()
        t.knn_cov_host(qh, K_NN, EPS, out=outs, stream=stream)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            e2e_t.append(dt)
    e2e_total = sum(e2e_t)
    e2e_total = sharding.reduce_max(e2e_total, dev)
    e2e_value = n_all * len(e2e_t) / e2e_total
    assert torch.equal(outs[0], idx.cpu())
    copy_probe = copy_bandwidth(dev, stream, qh, qd, outs, (idx, d2, cov)) if rank == 0 else None

    extras = {}
    if rank == 0 and ws == 1 and not args.headline_only:
        t.close()
        t = None
        extras["batched"] = measure_c3(md, m, reps=10)
        extras["served"] = measure_c4(duration=args.served_duration, speeds=(("nominal", 1.0),
                                                                             ("saturated", 1e6)))

    base = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(q, m)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "c2_scan131k_vs_map2M_k20_eps1e-3", "n_queries": N, "map_points": MAP_POINTS,
                       "k": K_NN, "eps": EPS, "cell_size": info["cell_size"], "occupied_cells": info["ncells"],
                       "scans_per_step": R, "ms_per_scan": ms_per_scan,
                       "tuned": tuned or "defaults (no cached configuration)",
                       "l2": "flushed by a 256 MB write before every scan (outside the scan's events)",
                       "parallelism": f"queries sharded by scan, {ws} rank(s), no collective"},
            "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                           "max": lat[-1], "scans": len(lat)},
            "roofline": roof,
            "l2_traffic": l2,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 12 * N,
                    "d2h_bytes_per_step": N * (8 * K_NN + 24), "step": "one scan through pc_knn_cov_host",
                    "path": "page-locked buffers: q read and idx/d2/cov written in place by the search "
                            "(whole-line block writes per warp); `copies` times the staged-copy path's parts",
                    "copies": copy_probe},
            "issue_roofline": issue_roofline(ms_per_scan, clk,
                                             torch.cuda.get_device_properties(dev).multi_processor_count),
            "clocks": clk,
            "search_paths": {"queries": path_stats["queries"],
                             "warp_search_frac": path_stats["warp_search"] / max(1, path_stats["queries"]),
                             "exhaustive": path_stats["exhaustive"],
                             "candidates_per_query": path_stats.get("candidates", 0) / max(1, path_stats["queries"])},
            "gpu_launches": args.steps * R,
        }
        line.update(extras)
        if base is not None:
            line["cpu_baseline"] = base
        print(json.dumps(line), flush=True)
    if t is not None:
        t.close()
    if dist:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- other workloads
def _timed(fn, flush, reps, stream):
    """Median CUDA-event time (ms) of fn() on `stream`, L2 flushed before each."""
    import torch

    evs = []
    with torch.cuda.stream(stream):
        for _ in range(3):
            flush.fill_(1)
            fn()
        for _ in range(reps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            evs.append((a, b))
    stream.synchronize()
    v = sorted(x.elapsed_time(y) for x, y in evs)
    return v[len(v) // 2], v


def _line(metric, value, unit, ms, args, config, **extra):
    d = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
         "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
         "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config}
    d.update(extra)
    print(json.dumps(d), flush=True)


def run_c1(args):
    """Self-kNN of 8192 uniform points, k = 10 (the parity case), timed."""
    import torch

    from paper_2308_07173_gb300 import pc
    from paper_2308_07173_gb300 import workloads as W

    pc.load()
    p = W.uniform_box(8192, seed=1)
    pd = torch.from_numpy(p).cuda()
    t = pc.Target(pd)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    ms, _ = _timed(lambda: t.knn_cov(pd, 10, EPS, stream=s), flush, min(args.steps, 200), s)
    _line("query points/sec, self-kNN(k=10)+cov, 8192 uniform points", len(p) / (ms / 1e3), UNIT, ms,
          args, {"workload": "c1_uniform8192_self_k10"})
    return 0


def measure_c3(md, m, reps: int = 10, tuned: dict = None) -> dict:
    """64 scans of 20k-130k points against the 2M map: one batched launch (a
    warp per scan tile) replayed as a CUDA graph vs 64 sequential launches,
    with identical results asserted.  Uses the tuner's cached configuration
    for this map and batch when one exists, else the defaults."""
    import torch

    from paper_2308_07173_gb300 import autotune, pc
    from paper_2308_07173_gb300 import workloads as W

    scans = W.scan_batch(64, seed=4)
    dev = md.device
    qs = [torch.from_numpy(x).to(dev) for x in scans]
    npts = sum(len(q) for q in qs)
    if tuned is None:
        tuned = autotune.lookup(autotune.default_cache(), K_NN, md.shape[0], npts)
    t = autotune.apply(md, tuned) if tuned else pc.Target(md)
    info = t.info()
    bufs = [(q, torch.empty((len(q), K_NN), dtype=torch.int32, device=dev),
             torch.empty((len(q), K_NN), dtype=torch.float32, device=dev),
             torch.empty((len(q), 6), dtype=torch.float32, device=dev)) for q in qs]
    seq_out = [(torch.empty_like(b[1]), torch.empty_like(b[2]), torch.empty_like(b[3])) for b in bufs]
    s = torch.cuda.Stream()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def sequential():
        for (q, _, _, _), (i, d, c) in zip(bufs, seq_out):
            t.knn_cov(q, K_NN, EPS, i, d, c, stream=s)

    b = pc.Batch(t, bufs, K_NN, EPS)
    clocks = Clocks(dev.index or 0)
    clocks.start()
    ms_seq, _ = _timed(sequential, flush, reps, s)
    ms_bat, v_bat = _timed(lambda: b.run(s), flush, reps, s)
    clk = clocks.stop()
    same = all(torch.equal(x[1], y[0]) and torch.equal(x[2].view(torch.int32), y[1].view(torch.int32))
               and torch.equal(x[3].view(torch.int32), y[2].view(torch.int32)) for x, y in zip(bufs, seq_out))
    assert same, "batched results differ from sequential"
    roof = algorithmic_roofline(md, info, [x[1] for x in bufs], npts, K_NN, ms_bat)
    b.close()
    t.close()
    return {"workload": "c3_64scans_logu20k-130k_map2M_k20", "queries": npts, "value": npts / (ms_bat / 1e3),
            "unit": UNIT, "ms": ms_bat, "ms_p99": v_bat[min(len(v_bat) - 1, int(0.99 * len(v_bat)))],
            "form": "one launch over the scans' tile table, CUDA graph replay",
            "tuned": tuned or "defaults (no cached configuration)",
            "sequential": {"value": npts / (ms_seq / 1e3), "ms": ms_seq, "launches": 64},
            "speedup_vs_sequential": ms_seq / ms_bat, "identical_to_sequential": bool(same),
            "roofline": roof, "clocks": clk, "gpu_launches_per_step": 1}


def run_c3(args):
    import torch

    from paper_2308_07173_gb300 import pc
    from paper_2308_07173_gb300 import workloads as W

    pc.load()
    _, m = W.scan_vs_map(MAP_POINTS)
    md = torch.from_numpy(m).cuda()
    r = measure_c3(md, m, reps=min(args.steps, 50))
    ms = r.pop("ms")
    _line("query points/sec, 64-scan batch (20k-130k each) vs 2M map, kNN(k=20)+cov", r.pop("value"),
          r.pop("unit"), ms, args, {"workload": r.pop("workload"), "queries": r["queries"]},
          **r, gpu_launches=1)
    return 0


def measure_c4(duration: float, speeds, map_points: int = 5_000_000, warm_scans: int = 20,
               repeats: int = 3, clock_ms: int = 200, step_scans: int = 16, step_points: int = 1 << 20,
               slots: int = 3) -> dict:
    """Serving: Poisson scans from 8 vehicles x 3 LiDARs at 20 Hz (replayed
    `speed` times faster: the arrival rate scales by `speed`) against a
    resident map; continuous batching vs one host-buffer call per scan."""
    import torch

    from paper_2308_07173_gb300 import autotune, pc, serve
    from paper_2308_07173_gb300 import workloads as W

    tr = W.oval_1500()
    m = tr.sample_map(map_points, seed=5)
    md = torch.from_numpy(m).cuda()
    arr = W.arrival_stream(duration=duration, seed=5)
    reqs = serve.requests_from_arrivals(arr)
    npts = sum(r.n for r in reqs)
    tuned = autotune.lookup(autotune.default_cache(), K_NN, map_points, 0)
    t = autotune.apply(md, tuned) if tuned else pc.Target(md)
    serve.prepare(reqs)
    srv = serve.Server(t, K_NN, EPS, hbm_budget=2 << 30, max_step_scans=step_scans, slots=slots, in_place=True,
                       max_step_points=step_points)
    warm = serve.requests_from_arrivals(arr[:warm_scans])
    serve.prepare(warm)
    srv.serve(warm, speed=1e6)
    serve.serve_per_scan(t, K_NN, EPS, warm, speed=1e6)
    out = {"workload": f"c4_24lidars_20hz_poisson_map{map_points // 1_000_000}M_k20",
           "arrival_seconds": duration, "scans": len(reqs), "points": npts,
           "offered_points_per_s_at_1x": npts / duration, "hbm_budget_bytes": 2 << 30,
           "max_step_scans": step_scans, "max_step_points": step_points, "slots": slots,
           "tuned": tuned or "defaults (no cached configuration)",
           "io": "both forms read the page-locked scans and write page-locked results in place "
                 "(served: one batched launch per step; per-scan: pc_knn_cov_host per scan)"}
    for name, speed in speeds:
        # host-timed latencies: each rate is replayed `repeats` times, served
        # and per-scan in alternating order, and the medians over the replays
        # are compared (a shared host can stall one replay)
        # the sampler's driver queries stalled paced replays by 20-280 ms now
        # and then (none in replays without it), so it runs only while every
        # scan is queued at once, where the GPU is busy throughout
        sample = clock_ms > 0 and speed >= 1e5
        clocks = Clocks(torch.cuda.current_device(), interval_ms=clock_ms)
        if sample:
            clocks.start()
        runs = {"served": [], "per_scan": []}
        for rep in range(repeats):
            order = ("served", "per_scan") if rep % 2 == 0 else ("per_scan", "served")
            for who in order:
                if who == "served":
                    runs[who].append(srv.serve(reqs, speed=speed))
                else:
                    runs[who].append(serve.serve_per_scan(t, K_NN, EPS, reqs, speed=speed))
        clk = clocks.stop() if sample else {"sm_mhz": None, "reasons": [],
                                            "note": "not sampled during paced replays (see the saturated record)"}

        def med(who, key):
            return statistics.median(r[key] for r in runs[who])

        sv = {key: med("served", key) for key in ("p50_ms", "p99_ms", "throughput_pts_s", "mean_scans_per_step",
                                                    "steps", "wall_s")}
        ps = {key: med("per_scan", key) for key in ("p50_ms", "p99_ms", "throughput_pts_s", "wall_s")}
        out[name] = {"arrival_rate_multiple": speed if speed < 1e5 else "all at t=0", "replays": repeats,
                     "served": sv, "per_scan": ps, "served_runs": runs["served"], "per_scan_runs": runs["per_scan"],
                     "clocks": clk, "served_p99_over_per_scan": sv["p99_ms"] / ps["p99_ms"],
                     "served_throughput_over_per_scan": sv["throughput_pts_s"] / ps["throughput_pts_s"]}
    assert t.sync_status() == pc.PC_OK
    t.close()
    return out


def run_c4(args):
    """C4 with the arrival-rate sweep: 10 s of arrivals replayed at
    --lambdas multiples of the nominal 480 scans/s, plus all at once
    (saturated), served vs per-scan at each rate."""
    from paper_2308_07173_gb300 import pc

    pc.load()
    lams = [float(x) for x in args.lambdas.split(",") if x]
    speeds = [(f"x{l:g}", l) for l in lams] + [("saturated", 1e6)]
    r = measure_c4(args.duration, speeds, repeats=2)
    sat = r["saturated"]["served"]
    _line("sustained points/sec and p50/p99 scan latency, 24 LiDARs x 20 Hz vs resident 5M map, kNN(k=20)+cov",
          sat["throughput_pts_s"], UNIT, 1e3 * sat["wall_s"] / max(1, sat["steps"]), args,
          {"workload": r["workload"], "arrival_seconds": args.duration, "scans": r["scans"]}, serving=r)
    return 0


def run_c5(args):
    """Large-map stress: 20M-point 4 km track with pit structures, ~1M
    ray-cast queries, k = 32."""
    import torch

    from paper_2308_07173_gb300 import pc
    from paper_2308_07173_gb300 import workloads as W

    from paper_2308_07173_gb300 import autotune

    pc.load()
    q, m = W.stress()
    md = torch.from_numpy(m).cuda()
    k = 32
    tuned = autotune.lookup(autotune.default_cache(), k, len(m), len(q))
    cfg = dict(autotune.DEFAULT, **(tuned or {}))
    t = autotune.apply(md, cfg)
    qd = torch.from_numpy(q).cuda()
    idx = torch.empty((len(q), k), dtype=torch.int32, device="cuda")
    d2 = torch.empty((len(q), k), dtype=torch.float32, device="cuda")
    cov = torch.empty((len(q), 6), dtype=torch.float32, device="cuda")
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    out = {}
    for name, probe in (("per_query_start", 2), ("calibrated_start", 1)):
        t.set_tune(cfg["tile"], cfg["warps"], cfg["rho_scale"], 0, probe, cfg["slots"])
        clocks = Clocks(torch.cuda.current_device())
        clocks.start()
        ms, v = _timed(lambda: t.knn_cov(qd, k, EPS, idx, d2, cov, stream=s), flush, min(args.steps, 20), s)
        clk = clocks.stop()
        t.stats(reset=True, stream=s)
        t.knn_cov(qd, k, EPS, idx, d2, cov, stream=s)
        st = t.stats(reset=True, stream=s)
        assert t.sync_status(s) == pc.PC_OK
        out[name] = {"ms": ms, "value": len(q) / (ms / 1e3), "clocks": clk,
                     "warp_search_frac": st["warp_search"] / max(1, st["queries"]),
                     "exhaustive": st["exhaustive"], "candidates_per_query": st["candidates"] / max(1, st["queries"])}
    info = t.info()
    best = out["per_query_start"]
    roof = algorithmic_roofline(md, info, [idx], len(q), k, best["ms"])
    _line("query points/sec, 1M queries vs 20M-point map (4 km + pit lane), kNN(k=32)+cov",
          best["value"], UNIT, best["ms"], args,
          {"workload": "c5_map20M_pit_noise1cm_queries1M_k32", "queries": len(q), "map_points": len(m),
           "cell_size": info["cell_size"], "occupied_cells": info["ncells"],
           "tuned": tuned or "defaults (no cached configuration)",
           "start_radius": "per query, from the point count of the 27 cells around it (the target's default "
                           "on this map: its calibration saw an uneven density)"},
          roofline=roof, search_paths={"warp_search_frac": best["warp_search_frac"], "exhaustive": best["exhaustive"],
                                       "candidates_per_query": best["candidates_per_query"]},
          clocks=best["clocks"], calibrated_start=out["calibrated_start"], gpu_launches=1)
    return 0


def run_window(args):
    """The C2 scan against a sliding-window submap of the 2M-point map: the
    window of the race-line station nearest the scan (260 m x 260 m, all
    heights: the sensor's 120 m range plus margin), set on the resident grid
    with no rebuild; timed next to the same search over the whole map."""
    import numpy as np
    import torch

    from paper_2308_07173_gb300 import pc, windows
    from paper_2308_07173_gb300 import workloads as W

    pc.load()
    q, m = W.scan_vs_map(MAP_POINTS)
    N = len(q)
    md, qd = torch.from_numpy(m).cuda(), torch.from_numpy(q).cuda()
    t = pc.Target(md)
    idx = torch.empty((N, K_NN), dtype=torch.int32, device="cuda")
    d2 = torch.empty((N, K_NN), dtype=torch.float32, device="cuda")
    cov = torch.empty((N, 6), dtype=torch.float32, device="cuda")
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    rw = windows.RaceLineWindows.along(W.oval_1500(), spacing=10.0, half=(130.0, 130.0, float("inf")))
    reps = max(5, min(args.steps, 200))
    ms_full, _ = _timed(lambda: t.knn_cov(qd, K_NN, EPS, idx, d2, cov, stream=s), flush, reps, s)
    station = rw.apply(t, np.median(q, axis=0))
    lo, hi = rw.window(station)
    lo_t, hi_t = torch.tensor(lo, device="cuda"), torch.tensor(hi, device="cuda")
    in_win = int(((md >= lo_t) & (md <= hi_t)).all(1).sum())
    q_out = int((~((qd >= lo_t) & (qd <= hi_t)).all(1)).sum())
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    ms, all_ms = _timed(lambda: t.knn_cov(qd, K_NN, EPS, idx, d2, cov, stream=s), flush, reps, s)
    clk = clocks.stop()
    st = t.sync_status(s)
    assert st == pc.PC_OK, pc.pc_status_string(st)
    ui = torch.unique(idx.view(-1).long())
    U_p = int(ui.numel())
    info = t.info()
    o = torch.tensor(info["origin"], device="cuda")
    cells = torch.floor((md[ui] - o) * (1.0 / info["cell_size"])).long()
    U_c = int(torch.unique((cells[:, 0] << 42) | (cells[:, 1] << 21) | cells[:, 2]).numel())
    alg = N * (12 + 8 * K_NN + 24) + 12 * U_p + 8 * U_c
    peak, kind = peaks()
    ach = alg / (ms / 1e3) / 1e9
    _line("query points/sec for kNN(k=20)+cov against a 260 m sliding-window submap of the 2M map", N / (ms / 1e3),
          UNIT, ms, args, {"workload": "window_c2_scan131k_map2M_win260m_k20", "n_queries": N,
                           "map_points": MAP_POINTS, "window_points": in_win, "queries_outside_window": q_out,
                           "station": station,
                           "l2": "flushed by a 256 MB write before every timed call"},
          roofline={"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                    "traffic": None, "peak_source": kind, "algorithmic_bytes": alg, "U_p": U_p, "U_c": U_c,
                    "kernel": "k_knn<0,true,true> (window variant)"},
          whole_map_ms=ms_full, latency_ms={"p50": all_ms[len(all_ms) // 2], "max": all_ms[-1]}, clocks=clk,
          gpu_launches=reps)
    t.close()
    return 0


def run_kernel(args):
    """The C2 workload with the covariance weighted by the Laplacian kernel
    descriptor (Table I; the paper's best), sigma = 0.1 m, fused into the
    search like the plain covariance; timed next to the plain fused search."""
    import torch

    from paper_2308_07173_gb300 import pc
    from paper_2308_07173_gb300 import workloads as W

    pc.load()
    q, m = W.scan_vs_map(MAP_POINTS)
    N = len(q)
    md, qd = torch.from_numpy(m).cuda(), torch.from_numpy(q).cuda()
    t = pc.Target(md)
    idx = torch.empty((N, K_NN), dtype=torch.int32, device="cuda")
    d2 = torch.empty((N, K_NN), dtype=torch.float32, device="cuda")
    cov = torch.empty((N, 6), dtype=torch.float32, device="cuda")
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    reps = max(5, min(args.steps, 200))
    ms_plain, _ = _timed(lambda: t.knn_cov(qd, K_NN, EPS, idx, d2, cov, stream=s), flush, reps, s)
    t.set_cov_kernel("laplacian", sigma=0.1)
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    ms, all_ms = _timed(lambda: t.knn_cov(qd, K_NN, EPS, idx, d2, cov, stream=s), flush, reps, s)
    clk = clocks.stop()
    st = t.sync_status(s)
    assert st == pc.PC_OK, pc.pc_status_string(st)
    alg = N * (12 + 8 * K_NN + 24)
    peak, kind = peaks()
    ach = alg / (ms / 1e3) / 1e9
    _line("query points/sec for kNN(k=20) + Laplacian-weighted cov, 131k scan vs 2M map", N / (ms / 1e3), UNIT, ms,
          args, {"workload": "kernel_laplacian_c2_scan131k_map2M_k20", "n_queries": N, "map_points": MAP_POINTS,
                 "sigma": 0.1, "l2": "flushed by a 256 MB write before every timed call"},
          roofline={"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                    "traffic": None, "peak_source": kind, "algorithmic_bytes_queries_only": alg,
                    "kernel": "k_knn<0,1,0> (weighted covariance fused)"},
          plain_fused_ms=ms_plain, latency_ms={"p50": all_ms[len(all_ms) // 2], "max": all_ms[-1]}, clocks=clk,
          gpu_launches=reps)
    t.close()
    return 0


def run_wall(args):
    """Wall detection (Sec. III-D) on a 131k-point body-frame ray-cast scan:
    voxel filter (0.2 m), 2-D vote ground filter, Euclidean clustering
    (0.45 m) and the wall's quadratic fit; one call per step, eager and as a
    replayed CUDA graph (the call allocates nothing)."""
    import torch

    from paper_2308_07173_gb300 import pc
    from paper_2308_07173_gb300 import workloads as W

    pc.load()
    pts = W.body_frame_scan(s0=130.0, w0=2.0, seed=130)
    N = len(pts)
    pd = torch.from_numpy(pts).cuda()
    w = pc.WallDetector(N)
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    reps = max(5, min(args.steps, 200))
    ms_eager, _ = _timed(lambda: w.detect(pd, stream=s), flush, reps, s)
    res = w.result(stream=s)
    assert res["status"] == pc.PC_OK and res["wall_label"] >= 0
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin(capture_error_mode="thread_local")
        w.detect(pd, stream=s)
        g.capture_end()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    ms, all_ms = _timed(lambda: g.replay(), flush, reps, s)
    clk = clocks.stop()
    r2 = w.result(stream=s)
    assert r2["beta"] == res["beta"]
    w.close()
    alg = 12 * N
    peak, kind = peaks()
    _line("body-frame scan points/sec through wall detection (voxel, 2-D vote, clustering, fit)", N / (ms / 1e3),
          UNIT, ms, args, {"workload": "wall_body_scan131k_voxel0.2_tol0.45", "n_points": N,
                           "n_voxels": res["n_voxels"], "n_vertical": res["n_vertical"],
                           "wall_count": res["wall_count"], "d_w": res["d_w"],
                           "l2": "flushed by a 256 MB write before every timed call"},
          roofline={"bound": "hbm", "achieved": alg / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                    "frac": alg / (ms / 1e3) / 1e9 / peak, "traffic": None, "peak_source": kind,
                    "algorithmic_bytes_points_only": alg, "kernel": "pc_wall_detect (graph of ~40 launches)"},
          eager_ms=ms_eager, latency_ms={"p50": all_ms[len(all_ms) // 2], "max": all_ms[-1]}, clocks=clk,
          gpu_launches=reps)
    return 0


def run_append(args):
    """Incremental map update: the 2M-point map built from 1.8M points with
    200k appended (no main-grid rebuild), the C2 scan searched over the union
    (one launch visiting the main and the appended-points grids), next to the
    same search on a map built whole; also the append and compaction times."""
    import torch

    from paper_2308_07173_gb300 import pc
    from paper_2308_07173_gb300 import workloads as W

    pc.load()
    q, m = W.scan_vs_map(MAP_POINTS)
    N = len(q)
    md, qd = torch.from_numpy(m).cuda(), torch.from_numpy(q).cuda()
    n_main = MAP_POINTS - 200_000
    whole = pc.Target(md)
    t = pc.Target(md[:n_main].contiguous())
    s = torch.cuda.Stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t.append(md[n_main:].contiguous(), stream=s)
    s.synchronize()
    append_ms = (time.perf_counter() - t0) * 1e3
    idx = torch.empty((N, K_NN), dtype=torch.int32, device="cuda")
    d2 = torch.empty((N, K_NN), dtype=torch.float32, device="cuda")
    cov = torch.empty((N, 6), dtype=torch.float32, device="cuda")
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    reps = max(5, min(args.steps, 200))
    ms_whole, _ = _timed(lambda: whole.knn_cov(qd, K_NN, EPS, idx, d2, cov, stream=s), flush, reps, s)
    ref = idx.clone()
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    ms, all_ms = _timed(lambda: t.knn_cov(qd, K_NN, EPS, idx, d2, cov, stream=s), flush, reps, s)
    clk = clocks.stop()
    assert t.sync_status(s) == pc.PC_OK
    assert torch.equal(ref, idx)
    t0 = time.perf_counter()
    t.compact(stream=s)
    s.synchronize()
    compact_ms = (time.perf_counter() - t0) * 1e3
    alg = N * (12 + 8 * K_NN + 24)
    peak, kind = peaks()
    _line("query points/sec for kNN(k=20)+cov over a 2M map grown by 200k appended points", N / (ms / 1e3), UNIT,
          ms, args, {"workload": "append_c2_scan131k_map1.8M_plus200k_k20", "n_queries": N, "map_main": n_main,
                     "appended": MAP_POINTS - n_main, "l2": "flushed by a 256 MB write before every timed call"},
          roofline={"bound": "hbm", "achieved": alg / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                    "frac": alg / (ms / 1e3) / 1e9 / peak, "traffic": None, "peak_source": kind,
                    "algorithmic_bytes_queries_only": alg, "kernel": "k_knn_union<0,1,0> (main + appended grids)"},
          whole_map_ms=ms_whole, append_ms=append_ms, compact_ms=compact_ms,
          latency_ms={"p50": all_ms[len(all_ms) // 2], "max": all_ms[-1]}, clocks=clk, gpu_launches=reps)
    t.close()
    whole.close()
    return 0


def run_gicp(args):
    """GICP on the C2 scan (131k points) against the 2M-point map: one
    linearisation (exact nearest-point pairing within 1 m, the combined
    covariance and the 6x6 normal equations) per step, then a 10-iteration
    registration (linearise + device-side update) replayed as a CUDA graph."""
    import numpy as np
    import torch

    from paper_2308_07173_gb300 import gicp, pc
    from paper_2308_07173_gb300 import workloads as W

    pc.load()
    q, m = W.scan_vs_map(MAP_POINTS)
    N = len(q)
    md, qd = torch.from_numpy(m).cuda(), torch.from_numpy(q).cuda()
    s = torch.cuda.Stream()
    reg = gicp.Registration(md, k=K_NN, eps=EPS)
    scov = reg.source_covariances(qd)
    pose0 = np.concatenate([np.eye(3).ravel(), [0.05, -0.03, 0.01]]).astype(np.float32)
    pose = torch.from_numpy(pose0).cuda()
    out = torch.empty(29, dtype=torch.float64, device="cuda")
    corr = torch.empty(N, dtype=torch.int32, device="cuda")
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    t = reg.map
    t.gicp_linearize(reg.map_cov, qd, scov, pose, 1.0, out=out, corr=corr, stream=s)
    s.synchronize()
    assert t.sync_status(s) == pc.PC_OK
    pairs = int(out[28].item())
    used = corr[corr >= 0].long()
    U_p = int(torch.unique(used).numel())
    info = t.info()
    pts = md[torch.unique(used)]
    o = torch.tensor(info["origin"], device="cuda")
    cells = torch.floor((pts - o) * (1.0 / info["cell_size"])).long()
    U_c = int(torch.unique((cells[:, 0] << 42) | (cells[:, 1] << 21) | cells[:, 2]).numel())
    reps = max(5, min(args.steps, 200))
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    ms, all_ms = _timed(lambda: t.gicp_linearize(reg.map_cov, qd, scov, pose, 1.0, out=out, stream=s),
                        flush, reps, s)
    iters = 10
    p2 = torch.from_numpy(pose0).cuda()

    def align():
        p2.copy_(pose, non_blocking=True)
        reg.align(qd, scov, p2, iters=iters, max_dist=1.0, graph=True, stream=s)

    ms_reg, _ = _timed(align, flush, max(5, min(args.steps, 50)), s)
    clk = clocks.stop()
    assert t.sync_status(s) == pc.PC_OK
    # algorithmic bytes of one linearisation: the scan and its covariances,
    # the paired map covariances, the distinct map points and cells touched
    alg = N * (12 + 24) + pairs * 24 + 16 * U_p + 8 * U_c
    peak, kind = peaks()
    ach = alg / (ms / 1e3) / 1e9
    _line("source points/sec through one GICP linearisation (C2 scan vs 2M-point map)", N / (ms / 1e3), UNIT, ms,
          args, {"workload": "gicp_c2_scan131k_vs_map2M_maxdist1m", "n_points": N, "pairs": pairs,
                 "map_points": MAP_POINTS, "l2": "flushed by a 256 MB write before every timed call"},
          roofline={"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                    "traffic": None, "peak_source": kind, "algorithmic_bytes": alg, "U_p": U_p, "U_c": U_c,
                    "kernel": "k_gicp_linearize"},
          registration={"iterations": iters, "ms": ms_reg, "ms_per_iteration": ms_reg / iters,
                        "registrations_per_s": 1e3 / ms_reg, "graph": True},
          latency_ms={"p50": all_ms[len(all_ms) // 2], "max": all_ms[-1]}, clocks=clk,
          gpu_launches=reps)
    reg.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
