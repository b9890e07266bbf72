#!/usr/bin/env python3
"""Benchmark of the KS cutoff-table sweep on GB300.

Workload (one step = one pass of the whole path): the 90-cell table sweep,
exponents {1.5, 1.75, ..., 3.5} x sample sizes {10, 20, 50, 100, 200, 500,
1000, 2000, 5000, 10000}, xmin = 1, 100,000 replicates per cell: for every
replicate n Philox draws through the inverse-CDF table, the histogram, the
binary64 Newton fit, the KS distance, then the 90/95/99% order statistics
per cell.  9,000,000 replicates and 1.6992e10 draws per step.

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.
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

from paper_1305_6738_gb300 import inputs  # noqa: E402

Q = [0.90, 0.95, 0.99]
METRIC = "KS replicates/sec and samples/sec per (alpha,n) vs roofline; p50/p99 fit-request latency"

# Roofline of the dominant kernel (the sampler).  Algorithmic work per draw:
# a quarter of a Philox4x32-10 block (the draw's high word) = 10 rounds x 2
# products / 4 draws = 5 full 32x32->64-bit multiplies (plus ~10 XOR/ADD ops
# on the wider ALU pipe); the low word's block, drawn only for the rare draws
# whose interval of m holds a threshold or that lie beyond the table, is not
# counted.  The binding unit is the wide-multiply pipe: 32 lanes per SM per
# clock on GB300 (a quarter of the 128 FP32/ALU lanes; measured with an
# issue-rate probe), so the ceiling is SMs x 32 x clock / 5 draws per second.
MUL_PER_DRAW = 5
MUL_LANES_PER_SM = 32

# DRAM bytes per replicate of the sampler from one ncu capture (sweep at 33,000
# replicates per cell, 2.97e6 replicates in one wave: 1,090 MB in its three
# launches, mostly the replicate records written), keyed by the hash of the
# kernel sources it was taken on (reported as null once they change).  The
# bench scales it to a launch by the replicates per launch.
TRAFFIC_PER_REPLICATE = {"4104ca9b1f7015f2": (43.655168e6 + 62.887168e6 + 54.574848e6 + 768.936192e6 + 44.339456e6
                                              + 114.823424e6) / 2.97e6}


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ["pl_device.cuh", "pl_kernels.cu"]:
        with open(os.path.join(ROOT, "paper_1305_6738_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f)
    except OSError:
        return {}


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                       "-lms", "200", "-i", gpu_id], stdout=self.tmp,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r.strip().split(", ") for r in self.tmp.read().splitlines() if r.strip()]
        os.unlink(self.tmp.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1].split()[0]))
                smax.append(float(r[2].split()[0]))
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_query_id(device: int) -> str:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if device < len(ids):
            return ids[device]
    return str(device)


# ----------------------------------------------------------------------------- cpu
def cpu_oracle_rate(sample_reps: int, threads: int) -> dict:
    """The oracle as it stands, on sample_reps replicates of every cell, timed
    per cell and extrapolated linearly to the full replicate count."""
    import oracle
    oracle.build()
    sweep = inputs.cutoff_table_sweep()
    t_full = 0.0
    wall = 0.0
    for c in sweep:
        t0 = time.perf_counter()
        oracle.cell(c.alpha, c.xmin, c.n, sample_reps, seed=1, cell_id=c.cell_id, threads=threads)
        dt = time.perf_counter() - t0
        wall += dt
        t_full += dt / sample_reps * c.replicates
    total_R = sum(c.replicates for c in sweep)
    draws = sum(c.replicates * c.n for c in sweep)
    return {"value": total_R / t_full, "samples_per_s": draws / t_full, "wall_s": wall,
            "sample": f"{sample_reps} replicates of each of the 90 cells (draws, fit, KS, seed 1), "
                      f"timed per cell and extrapolated linearly to 100,000 replicates per cell"}


# ----------------------------------------------------------------------------- serving
SERVE_B = 2500
SERVE_RATE = 200.0
SERVE_BUDGET = 40 << 30


def serving_config(args) -> dict:
    return {"workload": (f"serving: Poisson arrivals at {SERVE_RATE:.0f} fit requests/s, n log-uniform "
                         "[50, 1e6], alpha U(1.5, 3.5), xmin=1, 10% rounded-lognormal data; per request "
                         f"MLE, D and a {SERVE_B:,}-replicate bootstrap p-value; 40 GB device budget"),
            "rate_per_s": SERVE_RATE, "B": SERVE_B, "duration_s": args.duration,
            "warmup_s": args.serve_warmup, "budget_bytes": SERVE_BUDGET, "workers": args.workers,
            "precision_form": args.precision, "request_seed": 4, "bootstrap_seed": 1,
            "l2": "inputs larger than L2 in aggregate (requests of up to 4 MB stream through)",
            "parallelism": "one GPU, requests overlapped on per-worker streams"}


def request_data_lognormal(r):
    import numpy as np
    return inputs.rounded_lognormal(np.random.default_rng((44, r.request_id)), r.n)


def serving_cpu_baseline(reqs, threads: int) -> dict:
    """The oracle's bootstrap on a bounded sample of the request stream: 32
    requests spread evenly over it (their data drawn by the oracle's sampler, the same integers the
    library's sampler gives), timed with b1 and b2 replicates and extrapolated
    linearly to B (the data fit is the intercept)."""
    import numpy as np
    import oracle
    oracle.build()
    picks = reqs[::max(1, len(reqs) // 32)][:32]
    b1, b2 = threads, 3 * threads
    per = []
    wall = 0.0
    for r in picks:
        if r.lognormal:
            x = request_data_lognormal(r)
        else:
            x = inputs.as_request_data(oracle.sample(r.alpha, r.xmin, 4, r.request_id, 0,
                                                     inputs.PURPOSE_TESTDATA, r.n))
        t = []
        for b in (b1, b2):
            t0 = time.perf_counter()
            oracle.bootstrap_pvalue(x, r.xmin, b, 1, r.request_id, threads)
            t.append(time.perf_counter() - t0)
        wall += sum(t)
        slope = max(0.0, (t[1] - t[0]) / (b2 - b1))
        per.append(t[0] + slope * (SERVE_B - b1))
    return {"value": len(per) / sum(per), "p50_ms": 1e3 * statistics.median(per), "wall_s": wall,
            "sample": (f"{len(per)} requests spread evenly over the stream, oracle bootstrap timed at B={b1} "
                       f"and B={b2} and extrapolated linearly to B={SERVE_B}; requests served one at a time")}


def serving_data(reqs, pl, ctx, torch):
    """Host int32 data of the requests: power-law data from the library's
    sampler (stream tag 2, cell id = request id, seed 4), lognormal data from
    the input module; generated before the clock starts."""
    buf = torch.empty(max(r.n for r in reqs), dtype=torch.int64, device="cuda")
    data = []
    for r in reqs:
        if r.lognormal:
            data.append(request_data_lognormal(r))
            continue
        ctx.pl_sample(r.alpha, r.xmin, 4, r.request_id, inputs.PURPOSE_TESTDATA, 0, 1, r.n, buf)
        data.append(buf[:r.n].clamp(max=inputs.INT32_MAX).to(torch.int32).cpu().numpy())
    return data


def serve_measure(local: int, duration: float, warmup: float, workers: int, prec: int, pl, torch,
                  serve_log: str = "") -> dict:
    """Open-loop Poisson arrivals at SERVE_RATE for warmup + duration seconds
    through the serving engine; latency = done - scheduled arrival of the
    requests arriving after the warm-up."""
    import threading
    import numpy as np
    ctx = pl.Context(local)
    t0 = time.perf_counter()
    reqs = inputs.serving_requests(warmup + duration, SERVE_RATE, seed=4)
    data = serving_data(reqs, pl, ctx, torch)
    generate_s = time.perf_counter() - t0
    ctx.close()
    srv = pl.Server(local, SERVE_BUDGET, workers=workers, prec=prec, seed=1, B=SERVE_B)
    base = srv.pl_server_now() + 0.2
    lag = []

    def submit_all():
        for r, x in zip(reqs, data):
            dt = base + r.arrival_s - srv.pl_server_now()
            if dt > 0:
                time.sleep(dt)
            lag.append(srv.pl_server_now() - (base + r.arrival_s))
            srv.pl_server_submit(r.request_id, x, r.xmin)

    sampler = None
    results = {}
    th = threading.Thread(target=submit_all)
    th.start()
    max_queue = max_running = 0
    max_reserved = 0
    launches0 = None
    while len(results) < len(reqs):
        now = srv.pl_server_now()
        if sampler is None and now >= base + warmup:
            sampler = ClockSampler(gpu_query_id(local))
            launches0 = srv.pl_server_load()[3]
        for res in srv.pl_server_poll(256, 0.01):
            results[res["request_id"]] = res
        q, run, rb, _ = srv.pl_server_load()
        if sampler is not None:
            max_queue, max_running, max_reserved = max(max_queue, q), max(max_running, run), max(max_reserved, rb)
    th.join()
    clocks = sampler.stop() if sampler else {}
    launches = srv.pl_server_load()[3] - (launches0 or 0)
    srv.close()
    if serve_log:
        with open(serve_log, "w") as f:
            for r in reqs:
                res = results[r.request_id]
                f.write(json.dumps({"id": r.request_id, "n": r.n, "alpha": r.alpha, "lognormal": r.lognormal,
                                    "arrival_s": base + r.arrival_s, "submit_s": res["submit_s"],
                                    "start_s": res["start_s"], "done_s": res["done_s"],
                                    "status": res["status"], "alpha_hat": res["alpha_hat"],
                                    "p": res["p"]}) + "\n")
    timed = [r for r in reqs if r.arrival_s >= warmup]
    bad = [results[r.request_id]["status"] for r in timed if results[r.request_id]["status"] != 0]
    lat = np.array([results[r.request_id]["done_s"] - (base + r.arrival_s) for r in timed]) * 1e3
    wait = np.array([results[r.request_id]["start_s"] - results[r.request_id]["submit_s"] for r in timed]) * 1e3
    t_first = base + timed[0].arrival_s
    t_last = max(results[r.request_id]["done_s"] for r in timed)
    span = t_last - t_first
    big = np.array([r.n >= 100_000 for r in timed])
    return {"value": len(timed) / span, "timed": timed, "warmup_requests": len(reqs) - len(timed),
            "ms_per_request": 1e3 * span / len(timed), "generate_s": generate_s,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max()), "mean": float(lat.mean()),
                           "p50_n_ge_1e5": float(np.percentile(lat[big], 50)) if big.any() else None,
                           "p99_n_lt_1e5": float(np.percentile(lat[~big], 99)) if (~big).any() else None,
                           "queue_wait_p99": float(np.percentile(wait, 99)),
                           "submit_lag_p99": float(np.percentile(np.array(lag) * 1e3, 99))},
            "draws_per_s": sum(SERVE_B * r.n for r in timed) / span, "failed_requests": len(bad),
            "load": {"max_queued": max_queue, "max_running": max_running, "max_reserved_bytes": max_reserved},
            "h2d_bytes_per_request": statistics.mean(4 * r.n for r in timed),
            "launches": launches, "clocks": clocks}


def run_serving(args):
    threads = os.cpu_count() or 1
    config = serving_config(args)
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return
        reqs = inputs.serving_requests(args.serve_warmup + args.duration, SERVE_RATE, seed=4)
        cb = serving_cpu_baseline([r for r in reqs if r.arrival_s >= args.serve_warmup], threads)
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "requests/s",
                "n_gpus": 0, "steps": len(reqs), "warmup": 0, "ms_per_step": 1e3 / cb["value"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic request stream", "config": config,
                "cpu_baseline": {"value": cb["value"], "unit": "requests/s", "cores": threads,
                                 "kind": "oracle", "sample": cb["sample"]},
                "e2e": {"value": cb["value"], "unit": "requests/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return

    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_1305_6738_gb300 import pl
    prec = pl.PL_FP32_BULK if args.precision == "fp32-bulk" else pl.PL_FP64
    m = serve_measure(local, args.duration, args.serve_warmup, args.workers, prec, pl, torch, args.serve_log)
    config["generate_s"] = m["generate_s"]
    timed = m["timed"]
    line = {"metric": METRIC, "value": m["value"], "unit": "requests/s", "n_gpus": 1, "steps": len(timed),
            "warmup": m["warmup_requests"], "ms_per_step": m["ms_per_request"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if prec == pl.PL_FP32_BULK else "f64",
            "data": "synthetic request stream (library sampler, stream tag 2; rounded lognormal)",
            "config": config, "latency_ms": m["latency_ms"], "draws_per_s": m["draws_per_s"],
            "failed_requests": m["failed_requests"], "load": m["load"],
            "e2e": {"value": m["value"], "unit": "requests/s", "h2d_bytes_per_step": m["h2d_bytes_per_request"],
                    "d2h_bytes_per_step": 24,
                    "note": "the serving value is end to end: host data in, host results out"},
            "gpu_launches": m["launches"], "clocks": m["clocks"]}
    if not args.no_cpu_baseline:
        cb = serving_cpu_baseline(timed, threads)
        line["cpu_baseline"] = {"value": cb["value"], "unit": "requests/s", "cores": threads,
                                "kind": "oracle", "sample": cb["sample"], "p50_ms": cb["p50_ms"]}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- replicas
# ----------------------------------------------------------------------------- truncated law
TZ_WORKLOAD = ("Tables 2-6 run: truncated law on 1..K, K in {20,50,100,500,1000} x gamma in "
               "{0.25,...,4.0} (12) x N in {10,...,50000} (15), {R:,} replicates per cell, "
               "quantiles 0.9/0.95/0.99/0.999")


def tz_source_hash() -> str:
    h = hashlib.sha256()
    for f in ["pl_device.cuh", "pl_truncated.cuh", "pl_truncated.cu"]:
        with open(os.path.join(ROOT, "paper_1305_6738_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# DRAM bytes per replicate of the truncated replicate kernel from one
# one-pass ncu capture of a full Tables 2-6 launch (57.2 MB read + 148.3 MB
# written for 45,000,000 replicates: the 4-byte D of each replicate plus the
# tables), keyed by the hash of its sources (null once they change).
# The later keys are the same kernel after changes to pl_device.cuh that only
# touch the untruncated samplers (a larger guide table; the lane-finish spill
# limit and lane sizes, the lane-form sampler's limits, the shortened-histogram
# bound and the per-cell flags), which the truncated kernel does not use (it
# has its own constants and cells).
TZ_TRAFFIC_PER_REPLICATE = {"bb5f053fedd20812": (57234944 + 148284928) / 45e6,
                            "a2952dc4a133b7a3": (57234944 + 148284928) / 45e6,
                            "86ecba4b8d4d58e2": (57234944 + 148284928) / 45e6,
                            "1141582e0e9bcfe7": (57234944 + 148284928) / 45e6}


def tz_cpu_oracle_rate(cells, sample_reps: int, threads: int) -> dict:
    """The oracle as it stands on sample_reps replicates of every truncated
    cell, timed per cell and extrapolated linearly to the full replicate count."""
    import oracle
    oracle.build()
    t_full = wall = 0.0
    for c in cells:
        t0 = time.perf_counter()
        oracle.tz_cell(c.gamma, c.K, c.n, sample_reps, seed=1, cell_id=c.cell_id, threads=threads)
        dt = time.perf_counter() - t0
        wall += dt
        t_full += dt / sample_reps * c.replicates
    total_R = sum(c.replicates for c in cells)
    draws = sum(c.replicates * c.n for c in cells)
    return {"value": total_R / t_full, "samples_per_s": draws / t_full, "wall_s": wall,
            "sample": f"{sample_reps} replicates of each of the {len(cells)} cells (draws, fit, KS, seed 1), "
                      f"timed per cell and extrapolated linearly to {cells[0].replicates:,} replicates per cell"}


def run_truncated(args):
    """One run of Tables 2-6 per step through pl_ks_cutoffs_truncated."""
    tcells = inputs.tables2to6_cells(args.tz_replicates)
    QS = list(inputs.TZ_QUANTILES)
    total_R = sum(c.replicates for c in tcells)
    draws = sum(c.replicates * c.n for c in tcells)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    config = {"workload": TZ_WORKLOAD.replace("{R:,}", f"{args.tz_replicates:,}"), "cells": len(tcells), "replicates_per_step": total_R,
              "draws_per_step": draws, "precision_form": args.precision, "seed": 1, "quantiles": QS,
              "l2": "256 MiB buffer written between timed steps (L2 flush)",
              "parallelism": f"replicas x{args.gpus}"}
    threads = os.cpu_count() or 1
    samp = max(1, threads)
    if args.impl == "reference":
        if rank != 0:
            return
        tz_cpu_oracle_rate(tcells[:15], 1, threads)
        vals = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            vals.append(tz_cpu_oracle_rate(tcells, samp, threads))
        wall = time.perf_counter() - t0
        value = statistics.mean(v["value"] for v in vals)
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "replicates/s",
                "samples_per_s": statistics.mean(v["samples_per_s"] for v in vals), "n_gpus": 0,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total_R / value,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (Philox streams, seed 1)", "config": config,
                "cpu_baseline": {"value": value, "unit": "replicates/s", "cores": threads, "kind": "oracle",
                                 "sample": vals[0]["sample"]},
                "e2e": {"value": value, "unit": "replicates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "wall_s": wall}
        print(json.dumps(line), flush=True)
        return

    import numpy as np
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_1305_6738_gb300 import pl
    ctx = pl.Context(local)
    prec = pl.PL_FP32_BULK if args.precision == "fp32-bulk" else pl.PL_FP64
    seed = replica_seed(rank)
    cells = [pl.TCell(c.gamma, c.K, c.n, c.replicates, c.cell_id) for c in tcells]
    cut = torch.empty(len(cells) * len(QS), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def step():
        ctx.pl_ks_cutoffs_truncated(cells, seed, QS, prec, cutoffs=cut)

    ctx.pl_set_tracing(True)
    for _ in range(args.warmup):
        step()
    ctx.pl_sync()
    launches0 = ctx.pl_trace()["launches"]
    sampler = ClockSampler(gpu_query_id(local))
    barrier()
    step_ms, kern_ms, law_ms = [], [], []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        tr = ctx.pl_trace()
        step_ms.append(e0.elapsed_time(e1))
        kern_ms.append(tr["replicate_ms"])
        law_ms.append(tr["law_ms"])
    barrier()
    clocks = sampler.stop()
    launches = ctx.pl_trace()["launches"] - launches0
    ctx.pl_sync()
    total_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    value = job_rate(total_R * args.steps, world, total_ms / 1000.0)
    sps = job_rate(draws * args.steps, world, total_ms / 1000.0)
    e2e_s = []
    host_cut = np.zeros(len(cells) * len(QS))
    for _ in range(max(2, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.pl_ks_cutoffs_truncated(cells, seed, QS, prec, cutoffs=host_cut)
        e2e_s.append(time.perf_counter() - t0)
    e2e_value = job_rate(total_R, world, max_over_ranks(statistics.mean(e2e_s), dist, "cuda"))
    props = torch.cuda.get_device_properties(local)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz") or 2070.0)
    mul_peak = props.multi_processor_count * MUL_LANES_PER_SM * sm_max * 1e6 / 1e9
    kmean = statistics.mean(kern_ms)
    achieved = MUL_PER_DRAW * draws / (kmean / 1000.0) / 1e9
    h = tz_source_hash()
    roofline = {"bound": "alu", "achieved": achieved, "peak": mul_peak, "unit": "Gmul/s (32x32->64)",
                "frac": achieved / mul_peak,
                "traffic": (TZ_TRAFFIC_PER_REPLICATE[h] * total_R if h in TZ_TRAFFIC_PER_REPLICATE else None),
                "kernel": "tz_replicate_kernel", "kernel_ms_per_step": kmean, "launches_per_step": 1,
                "setup_ms_per_step": statistics.mean(law_ms),
                "peak_basis": f"{props.multi_processor_count} SMs x {MUL_LANES_PER_SM} multiply lanes x "
                              f"{sm_max:.0f} MHz (max SM clock of MEASURED_PEAKS.json); "
                              f"{MUL_PER_DRAW} multiplies per draw"}
    line = {"metric": METRIC, "value": value, "unit": "replicates/s", "samples_per_s": sps,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if prec == pl.PL_FP32_BULK else "f64",
            "data": "synthetic (Philox streams, seed 1)", "config": config,
            "e2e": {"value": e2e_value, "unit": "replicates/s", "h2d_bytes_per_step": len(cells) * 40 + len(QS) * 8,
                    "d2h_bytes_per_step": host_cut.nbytes},
            "gpu_launches": launches, "roofline": roofline, "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = tz_cpu_oracle_rate(tcells, samp, threads)
        line["cpu_baseline"] = {"value": cb["value"], "unit": "replicates/s", "cores": threads,
                                "kind": "oracle", "sample": cb["sample"], "samples_per_s": cb["samples_per_s"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- bespoke cutoffs
BESPOKE_R = 10_000
BESPOKE_Q = [0.90, 0.95, 0.99]
LOOKUPS = 1_000_000


def bespoke_cpu_baseline(reqs, data, sample_reps: int, threads: int) -> dict:
    """The oracle composition per request (fit, D, the simulation at the
    fitted exponent and its quantiles) on sample_reps replicates, extrapolated
    linearly to BESPOKE_R replicates per request."""
    import numpy as np
    import oracle
    oracle.build()
    t_full = wall = 0.0
    for r, x in zip(reqs, data):
        xu = np.asarray(x, dtype=np.uint64)
        t0 = time.perf_counter()
        if r.truncated:
            g = oracle.tz_mle(xu, r.xmin_or_K)
            oracle.tz_ks(xu, r.xmin_or_K, g)
            t1 = time.perf_counter()
            oracle.tz_cell(g, r.xmin_or_K, r.n, sample_reps, seed=1, cell_id=r.request_id, purpose=1,
                           threads=threads)
        else:
            a = oracle.mle(xu, 1)
            oracle.ks(xu, 1, a)
            t1 = time.perf_counter()
            oracle.cell(a, 1, r.n, sample_reps, seed=1, cell_id=r.request_id, purpose=1, threads=threads)
        t2 = time.perf_counter()
        wall += t2 - t0
        t_full += (t1 - t0) + (t2 - t1) / sample_reps * BESPOKE_R
    return {"value": len(reqs) / t_full, "wall_s": wall,
            "sample": f"every request's fit and D, and {sample_reps} of its {BESPOKE_R:,} bespoke replicates "
                      f"(extrapolated linearly)"}


def bespoke_reference(args, reqs, threads):
    """The reference arm: the oracle's composition per request on the same
    data (the oracle's own samplers draw the identical values)."""
    import numpy as np
    import oracle
    oracle.build()
    data = []
    for r in reqs:
        if r.truncated:
            x = oracle.tz_sample(r.exponent, r.xmin_or_K, 4, r.request_id, 0, inputs.PURPOSE_TESTDATA, r.n)
        else:
            x = oracle.sample(r.exponent, 1, 4, r.request_id, 0, inputs.PURPOSE_TESTDATA, r.n)
        data.append(np.minimum(x, np.uint64(inputs.INT32_MAX)).astype(np.int64))
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(bespoke_cpu_baseline(reqs, data, max(1, threads), threads))
    wall = time.perf_counter() - t0
    value = statistics.mean(v["value"] for v in vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "requests/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * len(reqs) / value,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (power-law data from the method's sampler, stream tag 2)",
            "config": {"workload": f"bespoke cutoffs: {len(reqs)} data sets, {BESPOKE_R:,} replicates each"},
            "cpu_baseline": {"value": value, "unit": "requests/s", "cores": threads, "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": value, "unit": "requests/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)


def run_bespoke(args):
    """64 data sets per step, each through pl_bespoke_cutoffs(_truncated)."""
    reqs = inputs.bespoke_requests()
    threads = os.cpu_count() or 1
    if args.impl == "reference":
        if int(os.environ.get("RANK", "0")) == 0:
            bespoke_reference(args, reqs, threads)
        return
    import numpy as np
    import torch
    from paper_1305_6738_gb300 import pl
    config = {"workload": f"bespoke cutoffs: {len(reqs)} data sets (32 untruncated alpha~U(1.6,3), n in "
                          f"[1e2,1e4]; 32 truncated K in {{20,100,1000}}, gamma~U(0.25,3), n in [10,1e4]), "
                          f"{BESPOKE_R:,} simulated replicates each, q=0.9/0.95/0.99; plus {LOOKUPS:,} lookups "
                          f"in the Table 1 grid",
              "requests_per_step": len(reqs), "replicates_per_step": len(reqs) * BESPOKE_R,
              "draws_per_step": sum(r.n for r in reqs) * BESPOKE_R, "precision_form": args.precision,
              "l2": "inputs far below L2; calls synchronise (host outputs)", "parallelism": "one GPU"}
    ctx = pl.Context(0)
    prec = pl.PL_FP32_BULK if args.precision == "fp32-bulk" else pl.PL_FP64
    buf = torch.empty(max(r.n for r in reqs), dtype=torch.int64, device="cuda")
    data, dev = [], []
    for r in reqs:
        if r.truncated:
            ctx.pl_sample_truncated(r.exponent, r.xmin_or_K, 4, r.request_id, inputs.PURPOSE_TESTDATA, 0, 1, r.n,
                                    buf)
        else:
            ctx.pl_sample(r.exponent, 1, 4, r.request_id, inputs.PURPOSE_TESTDATA, 0, 1, r.n, buf)
        x = buf[:r.n].clamp(max=inputs.INT32_MAX).to(torch.int32)
        dev.append(x.clone())
        data.append(x.cpu().numpy())
    pinned = [torch.from_numpy(x).pin_memory() for x in data]

    def one(r, x):
        if r.truncated:
            return ctx.pl_bespoke_cutoffs_truncated(x, r.xmin_or_K, BESPOKE_R, 1, r.request_id, BESPOKE_Q, prec)
        return ctx.pl_bespoke_cutoffs(x, 1, BESPOKE_R, 1, r.request_id, BESPOKE_Q, prec)

    for _ in range(args.warmup):
        for r, x in zip(reqs, dev):
            one(r, x)
    launches0 = ctx.pl_trace()["launches"]
    sampler = ClockSampler(gpu_query_id(0))
    torch.cuda.synchronize()
    step_s, lat = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for r, x in zip(reqs, dev):
            t1 = time.perf_counter()
            one(r, x)
            lat.append(time.perf_counter() - t1)
        step_s.append(time.perf_counter() - t0)
    clocks = sampler.stop()
    launches = ctx.pl_trace()["launches"] - launches0
    total_s = sum(step_s)
    value = len(reqs) * args.steps / total_s
    draws = config["draws_per_step"]
    # end to end: each request's data copied from pinned host memory inside the timed region
    e2e = []
    for _ in range(max(1, args.steps // 2)):
        t0 = time.perf_counter()
        for r, h in zip(reqs, pinned):
            one(r, h.to("cuda", non_blocking=True))
        e2e.append(time.perf_counter() - t0)
    e2e_value = len(reqs) / statistics.mean(e2e)
    # the untruncated requests again through one batched call (one simulation plan)
    un = [(r, x) for r, x in zip(reqs, dev) if not r.truncated]
    bx, bxm, bid = [x for _, x in un], [1] * len(un), [r.request_id for r, _ in un]
    ctx.pl_bespoke_cutoffs_batch(bx, bxm, BESPOKE_R, 1, bid, BESPOKE_Q, prec)
    batch_s = []
    for _ in range(max(2, args.steps)):
        t0 = time.perf_counter()
        ctx.pl_bespoke_cutoffs_batch(bx, bxm, BESPOKE_R, 1, bid, BESPOKE_Q, prec)
        batch_s.append(time.perf_counter() - t0)
    batched_line = {"requests": len(un), "requests_per_s": len(un) / statistics.mean(batch_s),
                    "ms_per_call": 1000 * statistics.mean(batch_s)}
    # lookups in a tabulated grid (Table 1's exponents and sizes, 2,000 replicates per cell)
    GA, GN = list(inputs.TABLE1_GAMMAS), list(inputs.TABLE1_NS)
    cells = [pl.Cell(a, 1, n, 2000, 100 * i + k) for i, a in enumerate(GA) for k, n in enumerate(GN)]
    table = torch.empty(len(cells) * len(BESPOKE_Q), dtype=torch.float64, device="cuda")
    ctx.pl_ks_cutoffs(cells, 1, BESPOKE_Q, prec, cutoffs=table)
    g = torch.Generator(device="cpu").manual_seed(8)
    qa = (1.25 + 2.75 * torch.rand(LOOKUPS, generator=g, dtype=torch.float64)).cuda()
    qn = torch.exp(math.log(10) + (math.log(50000) - math.log(10)) * torch.rand(LOOKUPS, generator=g,
                                                                               dtype=torch.float64)).long().cuda()
    out = torch.empty(LOOKUPS * len(BESPOKE_Q), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(3):
        ctx.pl_cutoff_lookup(GA, GN, table, len(BESPOKE_Q), qa, qn, out)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(10):
        ctx.pl_cutoff_lookup(GA, GN, table, len(BESPOKE_Q), qa, qn, out)
    e1.record(stream)
    torch.cuda.synchronize()
    lk_ms = e0.elapsed_time(e1) / 10
    lk_bytes = LOOKUPS * (8 + 8 + 8 * len(BESPOKE_Q))
    # lower end by KS minimisation on a large data set: a flat body below 10 and a
    # power law (alpha = 2.5) from 10, 10^6 values, the smallest 1,000 distinct
    # values as candidates
    rngx = np.random.default_rng(12)
    tail = torch.empty(700_000, dtype=torch.int64, device="cuda")
    ctx.pl_sample(2.5, 10, 4, 9999, inputs.PURPOSE_TESTDATA, 0, 1, 700_000, tail)
    xm_host = np.concatenate([rngx.integers(1, 10, 300_000),
                              tail.clamp(max=inputs.INT32_MAX).cpu().numpy()]).astype(np.int32)
    xm_dev = torch.from_numpy(xm_host).cuda()
    ctx.pl_estimate_xmin(xm_dev, 1000, 10)
    xm_s = []
    for _ in range(3):
        t0 = time.perf_counter()
        xm_res = ctx.pl_estimate_xmin(xm_dev, 1000, 10)
        xm_s.append(time.perf_counter() - t0)
    xmin_line = {"n": int(xm_host.size), "candidates": xm_res["candidates"], "estimate": xm_res["xmin"],
                 "alpha_hat": xm_res["alpha_hat"], "ms_per_estimate": 1000 * statistics.mean(xm_s)}
    if not args.no_cpu_baseline:
        import oracle
        oracle.build()
        t0 = time.perf_counter()
        oracle.estimate_xmin(xm_host.astype(np.uint64), 1000, 10, threads=threads)
        xmin_line["cpu_baseline_ms"] = 1000 * (time.perf_counter() - t0)
        xmin_line["cpu_cores"] = threads
    peaks = measured_peaks()
    hbm = float(peaks.get("hbm_gbs") or 6800.0)
    props = torch.cuda.get_device_properties(0)
    sm_max = float(peaks.get("sm_max_mhz") or 2070.0)
    mul_peak = props.multi_processor_count * MUL_LANES_PER_SM * sm_max * 1e6 / 1e9
    achieved = MUL_PER_DRAW * draws * args.steps / total_s / 1e9
    lat.sort()
    line = {"metric": METRIC, "value": value, "unit": "requests/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if prec == pl.PL_FP32_BULK else "f64",
            "data": "synthetic (power-law data from the method's sampler, stream tag 2)", "config": config,
            "replicates_per_s": value * BESPOKE_R, "samples_per_s": draws * args.steps / total_s,
            "latency_ms": {"p50": 1000 * lat[len(lat) // 2], "p99": 1000 * lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                           "max": 1000 * lat[-1]},
            "e2e": {"value": e2e_value, "unit": "requests/s",
                    "h2d_bytes_per_step": sum(4 * r.n for r in reqs),
                    "d2h_bytes_per_step": len(reqs) * (3 + len(BESPOKE_Q)) * 8},
            "gpu_launches": launches,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": mul_peak, "unit": "Gmul/s (32x32->64)",
                         "frac": achieved / mul_peak, "traffic": None,
                         "kernel": "whole step (sampler, finisher and truncated replicate kernels, host gaps included)",
                         "peak_basis": f"{props.multi_processor_count} SMs x {MUL_LANES_PER_SM} multiply lanes x "
                                       f"{sm_max:.0f} MHz; {MUL_PER_DRAW} multiplies per draw"},
            "lookup": {"queries_per_s": LOOKUPS / (lk_ms / 1000), "kernel_ms": lk_ms,
                       "roofline": {"bound": "hbm", "achieved": lk_bytes / (lk_ms / 1000) / 1e9, "peak": hbm,
                                    "unit": "GB/s", "frac": lk_bytes / (lk_ms / 1000) / 1e9 / hbm,
                                    "traffic": None,
                                    "note": "algorithmic bytes: query (16 B) in, nq cutoffs out; the kernel is "
                                            "bound by binary64 arithmetic (one log and two divisions per query), "
                                            "not by memory"}},
            "xmin_estimate": xmin_line,
            "batched_untruncated": batched_line,
            "clocks": clocks}
    if not args.no_cpu_baseline:
        cb = bespoke_cpu_baseline(reqs, data, max(1, threads), threads)
        line["cpu_baseline"] = {"value": cb["value"], "unit": "requests/s", "cores": threads, "kind": "oracle",
                                "sample": cb["sample"]}
    print(json.dumps(line), flush=True)
    ctx.close()


def cell_line(alpha: float, n: int, R: int, step_ms: float, sample_ms: float, finish_ms: float,
              mul_peak_gmul: float, f64_peak_gflops: float | None = None) -> dict:
    """One (alpha, n) cell run alone: replicates/s and samples/s over the
    call's device time, the sampler's fraction of the multiply-pipe peak, the
    finisher's time per replicate and the finisher's binary64 fraction (the
    fit's binary64 operations per replicate over the binary64 peak)."""
    draws = R * n
    fit_ops = FINISHER_NCU.get(kernel_source_hash(), {}).get("fit_f64_ops")
    return {"alpha": alpha, "n": n, "replicates": R, "ms": step_ms,
            "replicates_per_s": R / (step_ms / 1e3), "samples_per_s": draws / (step_ms / 1e3),
            "sampler_ms": sample_ms, "finisher_ms": finish_ms,
            "finisher_ns_per_replicate": finish_ms * 1e6 / R,
            "sampler_frac": (MUL_PER_DRAW * draws / (sample_ms / 1e3) / 1e9 / mul_peak_gmul
                             if sample_ms > 0 else None),
            "finisher_fp64_frac": (fit_ops * R / (finish_ms / 1e3) / 1e9 / f64_peak_gflops
                                   if fit_ops and f64_peak_gflops and finish_ms > 0 else None)}


def per_cell_rates(ctx, cells, seed: int, qs, prec: int, mul_peak_gmul: float, flush, torch,
                   reps: int = 3, f64_peak_gflops: float | None = None) -> list:
    """Every cell of the sweep run alone (its own call, after one warm-up
    call): the median over `reps` timed calls, each after an L2 flush, with
    CUDA events on the call's stream and the library's per-kernel trace."""
    stream = torch.cuda.current_stream()
    one_cut = torch.empty(len(qs), dtype=torch.float64, device="cuda")
    ctx.pl_set_tracing(True)
    rows = []
    for c in cells:
        ctx.pl_ks_cutoffs([c], seed, qs, prec, cutoffs=one_cut)
        ms, sm, fm = [], [], []
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.pl_ks_cutoffs([c], seed, qs, prec, cutoffs=one_cut)
            e1.record(stream)
            tr = ctx.pl_trace()  # synchronises
            ms.append(e0.elapsed_time(e1))
            sm.append(tr["sample_ms"])
            fm.append(tr["finish_ms"])
        rows.append(cell_line(c.alpha, c.n, c.replicates, statistics.median(ms), statistics.median(sm),
                              statistics.median(fm), mul_peak_gmul, f64_peak_gflops))
    return rows


# Finisher figures from one ncu capture of the sweep at 33,000 replicates per
# cell (FP32-bulk; from 32,768 replicates a cell takes the long lanes, as at
# full size), keyed by the hash of the kernel sources they were taken on
# (reported as null once the sources change): DRAM bytes read per replicate
# (its replicate records) and binary64 operations per replicate (DFMA counted
# as two, DADD and DMUL as one), mostly the fit.
FINISHER_NCU = {"4104ca9b1f7015f2": {
    "dram_read_per_replicate": 2154.135296e6 / 2.97e6,
    "f64_ops_per_replicate": (231.771286e6 + 170.849080e6 + 2 * 146.157496e6) / 2.97e6,
    # one alpha = 3.5, n = 10 cell of 200,000 replicates (no spills, trivial KS): the fit alone
    "fit_f64_ops": (4.806451e6 + 2.804522e6 + 2 * 6.206738e6) / 200000}}
ALGO_BYTES_PER_REPLICATE = 16  # D (binary32 or binary64) and alpha-hat (binary64) out


def finisher_roofline(fin_ms: float, total_R: int, waves: int, f64_peak_gflops: float, probe: dict) -> dict:
    """The finisher's binary64 fraction and its record traffic per replicate."""
    ncu = FINISHER_NCU.get(kernel_source_hash())
    out = {"kernel": "finish_kernel", "bound": "fp64", "ms_per_step": fin_ms,
           "ns_per_replicate": fin_ms * 1e6 / total_R, "launches_per_step": waves,
           "peak": 2.0 * f64_peak_gflops, "unit": "Gflop/s (binary64)",
           "peak_basis": (f"{probe['sms']} SMs x {probe['dfma_per_sm_clk']:.2f} binary64 FMA per SM per clock "
                          "(pl_probe_rates) x max SM clock x 2"),
           "algorithmic_bytes_per_replicate": ALGO_BYTES_PER_REPLICATE}
    if ncu:
        achieved = ncu["f64_ops_per_replicate"] * total_R / (fin_ms / 1e3) / 1e9
        out.update({"binary64_ops_per_replicate": ncu["f64_ops_per_replicate"], "achieved": achieved,
                    "frac": achieved / out["peak"],
                    "record_bytes_per_replicate": ncu["dram_read_per_replicate"]})
    else:
        out.update({"binary64_ops_per_replicate": None, "achieved": None, "frac": None,
                    "record_bytes_per_replicate": None})
    return out


def timed_calls(call, flush, torch, stream, steps: int, warmup: int) -> list:
    """CUDA-event milliseconds of `steps` calls on `stream`, each after an L2 flush."""
    for _ in range(warmup):
        call()
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms


def fp64_form_record(ctx, cells, seed: int, qs, flush, torch, stream, pl, value_f32: float) -> dict:
    """The same sweep in the binary64 form (fit, KS and sums all binary64)."""
    cut = torch.empty(len(cells) * len(qs), dtype=torch.float64, device="cuda")
    ms = timed_calls(lambda: ctx.pl_ks_cutoffs(cells, seed, qs, pl.PL_FP64, cutoffs=cut), flush, torch, stream,
                     steps=3, warmup=1)
    ctx.pl_set_tracing(True)
    ctx.pl_ks_cutoffs(cells, seed, qs, pl.PL_FP64, cutoffs=cut)
    tr = ctx.pl_trace()
    R = sum(c.replicates for c in cells)
    v = R / (statistics.mean(ms) / 1e3)
    return {"value": v, "unit": "replicates/s", "ms_per_step": statistics.mean(ms), "steps": len(ms),
            "sampler_ms": tr["sample_ms"], "finisher_ms": tr["finish_ms"],
            "fp32_bulk_over_fp64": value_f32 / v}


def c0_fp64_record(ctx, flush, torch, stream, pl) -> dict:
    """The plain method in binary64: alpha = 2.5, xmin = 1, n = 100, 10,000
    replicates, seed 1; device-resident cutoffs, and end to end with the host
    cell table in and host cutoffs out."""
    import numpy as np
    c = inputs.cutoff_cell_small()[0]
    cells = [pl.Cell(c.alpha, c.xmin, c.n, c.replicates, c.cell_id)]
    cut = torch.empty(len(Q), dtype=torch.float64, device="cuda")
    ms = timed_calls(lambda: ctx.pl_ks_cutoffs(cells, 1, Q, pl.PL_FP64, cutoffs=cut), flush, torch, stream,
                     steps=20, warmup=3)
    host = np.zeros(len(Q))
    e2e = []
    for _ in range(10):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.pl_ks_cutoffs(cells, 1, Q, pl.PL_FP64, cutoffs=host)
        e2e.append(time.perf_counter() - t0)
    return {"workload": "alpha=2.5, xmin=1, n=100, 10,000 replicates, seed 1, binary64 form",
            "value": c.replicates / (statistics.median(ms) / 1e3), "unit": "replicates/s",
            "ms_per_step": statistics.median(ms), "steps": len(ms),
            "e2e": {"value": c.replicates / statistics.median(e2e), "unit": "replicates/s",
                    "h2d_bytes_per_step": 40 + 8 * len(Q), "d2h_bytes_per_step": 8 * len(Q)},
            "cutoffs": host.tolist()}


def replica_seed(rank: int) -> int:
    """Replicas (one process per GPU) draw independent Philox streams: the key
    is the base seed plus the rank.  No data crosses ranks."""
    return 1 + rank


def max_over_ranks(x: float, dist, device) -> float:
    """The slowest rank's value (the job's time); x itself without a group."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the job's time."""
    return world * units_per_rank / seconds


# ----------------------------------------------------------------------------- main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32-bulk", "fp64"], default="fp32-bulk")
    ap.add_argument("--cpu-sample", type=int, default=64, help="replicates per cell for the CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--replicates", type=int, default=100_000,
                    help="replicates per cell (smaller values for profiler captures only)")
    ap.add_argument("--workload", choices=["sweep", "small", "large-n", "batched", "serving", "table1",
                                           "truncated", "bespoke"],
                    default="sweep",
                    help="sweep: the 90-cell table (the benchmark line); small: alpha=2.5, n=100, "
                         "10,000 replicates; large-n: alpha=2, n=1e6, 10,000 replicates; batched: "
                         "4,096 uneven instances x 2,000 replicates in one graph-captured launch; "
                         "serving: Poisson fit requests at 200/s through the serving engine; "
                         "table1: one run of the paper's Table 1 (120 cells x 50,000 replicates); "
                         "truncated: one run of Tables 2-6 (truncated law, 900 cells x 50,000 replicates); "
                         "bespoke: 64 data sets (both laws), each fitted with its own cutoffs from 10,000 "
                         "simulated replicates, plus 10^6 lookups in a tabulated grid and one lower-end "
                         "estimate on 10^6 values")
    ap.add_argument("--no-per-cell", action="store_true",
                    help="sweep: skip timing every (alpha, n) cell alone (the per_cell list)")
    ap.add_argument("--no-extras", action="store_true",
                    help="sweep: skip the probe, the FP64-form sweep, the FP64 small cell and the short "
                         "serving run")
    ap.add_argument("--extras-serve-s", type=float, default=15.0,
                    help="sweep: measured seconds of the short serving run")
    ap.add_argument("--large-n-replicates", type=int, default=10_000,
                    help="large-n: replicates (smaller values for profiler captures only)")
    ap.add_argument("--sampler", choices=["inverse-cdf", "multinomial"], default="inverse-cdf",
                    help="sweep/small/large-n/table1: draw each value by the inverse CDF (default) or the "
                         "histogram by conditional binomials (pl_ks_cutoffs_multinomial)")
    ap.add_argument("--tz-replicates", type=int, default=50_000,
                    help="truncated: replicates per cell (smaller values for profiler captures only)")
    ap.add_argument("--duration", type=float, default=60.0, help="serving: measured seconds")
    ap.add_argument("--serve-warmup", type=float, default=5.0, help="serving: warm-up seconds")
    ap.add_argument("--workers", type=int, default=8, help="serving: engine worker slots")
    ap.add_argument("--serve-log", default="", help="serving: write per-request results (JSON lines)")
    args = ap.parse_args()
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "truncated":
        return run_truncated(args)
    if args.workload == "bespoke":
        return run_bespoke(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload == "sweep":
        sweep = inputs.cutoff_table_sweep(args.replicates)
        wname = ("KS cutoff-table sweep: alpha in {1.5,...,3.5} (9) x n in {10,...,10000} (10), "
                 f"xmin=1, {args.replicates:,} replicates per cell")
    elif args.workload == "small":
        sweep = inputs.cutoff_cell_small()
        wname = "single cell: alpha=2.5, xmin=1, n=100, 10,000 replicates"
    elif args.workload == "table1":
        sweep = inputs.table1_cells()
        wname = ("Table 1 run: gamma in {1.25,...,4.0} (8) x N in {10,...,50000} (15), xmin=1, "
                 "50,000 replicates per cell, quantiles 0.9/0.95/0.99/0.999")
    elif args.workload == "large-n":
        sweep = inputs.large_n_cell(args.large_n_replicates)
        wname = (f"large-n heavy tail: alpha=2.0, xmin=1, n=1,000,000, {args.large_n_replicates:,} replicates "
                 "(block form)")
    else:
        sweep = inputs.batched_instances()
        wname = ("batched uneven: 4,096 instances, n log-uniform [10,1e5], alpha U(1.6,3.2), "
                 "xmin in {1,2,5}, 2,000 replicates each; one plan, graph-captured launch, autotuned split, "
                 "work-item size and dense bins")
    QS = list(inputs.TABLE1_QUANTILES) if args.workload == "table1" else Q
    total_R = sum(c.replicates for c in sweep)
    draws = sum(c.replicates * c.n for c in sweep)
    config = {"workload": wname,
              "cells": len(sweep), "replicates_per_step": total_R, "draws_per_step": draws,
              "precision_form": args.precision, "seed": 1, "quantiles": QS,
              "l2": "256 MiB buffer written between timed steps (L2 flush)",
              "parallelism": f"replicas x{args.gpus}"}
    threads = os.cpu_count() or 1

    if args.impl == "reference":
        if rank != 0:
            return
        samp = max(1, args.cpu_sample // 4)
        for _ in range(args.warmup):
            cpu_oracle_rate(1, threads)
        vals = []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            r = cpu_oracle_rate(samp, threads)
            vals.append(r)
        wall = time.perf_counter() - t0
        value = statistics.mean(v["value"] for v in vals)
        sps = statistics.mean(v["samples_per_s"] for v in vals)
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "replicates/s",
                "samples_per_s": sps, "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1000.0 * total_R / value, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic (Philox streams, seed 1)",
                "config": config,
                "cpu_baseline": {"value": value, "unit": "replicates/s", "cores": threads, "kind": "oracle",
                                 "sample": vals[0]["sample"]},
                "e2e": {"value": value, "unit": "replicates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0},
                "wall_s": wall}
        print(json.dumps(line), flush=True)
        return

    import numpy as np
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_1305_6738_gb300 import pl
    ctx = pl.Context(local)
    prec = pl.PL_FP32_BULK if args.precision == "fp32-bulk" else pl.PL_FP64
    seed = replica_seed(rank)
    cells = [pl.Cell(c.alpha, c.xmin, c.n, c.replicates, c.cell_id) for c in sweep]
    cut = torch.empty(len(cells) * len(QS), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    graph = None
    if args.workload == "batched":
        # untimed set-up: autotuned warp/block split, plan (tables), graph capture
        t0 = time.perf_counter()
        tune = ctx.pl_autotune_cells(cells, prec, sample_replicates=max(c.replicates for c in cells))
        plan = ctx.pl_plan_cutoffs(cells, QS, prec)
        config["autotuned"] = {"split_n": tune["split"], "item_reps": tune["item_reps"],
                               "hist_shift": tune["hist_shift"],
                               "sample": "the whole workload, median of 3 calls per setting"}
        config["plan_ms"] = (time.perf_counter() - t0) * 1e3
        gstream = torch.cuda.Stream()
        with torch.cuda.stream(gstream):
            plan.run(seed, cut, stream=gstream)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        l0 = ctx.pl_trace()["launches"]
        with torch.cuda.graph(graph, stream=gstream):
            plan.run(seed, cut)
        torch.cuda.synchronize()
        kernels_per_replay = ctx.pl_trace()["launches"] - l0

    cutoffs_call = ctx.pl_ks_cutoffs_multinomial if args.sampler == "multinomial" else ctx.pl_ks_cutoffs
    if args.sampler == "multinomial":
        if args.workload == "batched":
            raise SystemExit("--sampler multinomial: not for the batched workload")
        config["sampler"] = "multinomial (conditional binomials, stream tag 3)"

    def step():
        if graph is not None:
            graph.replay()
        else:
            cutoffs_call(cells, seed, QS, prec, cutoffs=cut)

    ctx.pl_set_tracing(graph is None)
    for _ in range(args.warmup):
        step()
    ctx.pl_sync()
    launches0 = ctx.pl_trace()["launches"]

    sampler = ClockSampler(gpu_query_id(local))
    barrier()
    step_ms, kern_ms, fin_ms = [], [], []
    waves = slaunch = 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        tr = ctx.pl_trace()  # synchronises; kernel time from events on the call's stream
        step_ms.append(e0.elapsed_time(e1))
        if graph is None:
            kern_ms.append(tr["sample_ms"])
            fin_ms.append(tr["finish_ms"])
            waves, slaunch = tr["waves"], tr["sample_launches"]
    barrier()
    clocks = sampler.stop()
    launches = ctx.pl_trace()["launches"] - launches0
    if graph is not None:  # each replay launches the captured kernels
        launches = kernels_per_replay * args.steps
    ctx.pl_sync()
    total_ms = max_over_ranks(sum(step_ms), dist, "cuda")
    value = job_rate(total_R * args.steps, world, total_ms / 1000.0)
    sps = job_rate(draws * args.steps, world, total_ms / 1000.0)

    # end to end through the public call with host buffers: host cell table in,
    # host cutoffs out (the call copies and synchronises), wall clock
    e2e_s = []
    host_cut = np.zeros(len(cells) * len(QS))
    for _ in range(max(3, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cutoffs_call(cells, seed, QS, prec, cutoffs=host_cut)
        e2e_s.append(time.perf_counter() - t0)
    if graph is not None:  # trace one plain call for the per-kernel times
        ctx.pl_set_tracing(True)
        ctx.pl_ks_cutoffs(cells, seed, QS, prec, cutoffs=cut)
        tr = ctx.pl_trace()
        kern_ms, fin_ms = [tr["sample_ms"]], [tr["finish_ms"]]
        waves, slaunch = tr["waves"], tr["sample_launches"]
    e2e_value = job_rate(total_R, world, max_over_ranks(statistics.mean(e2e_s), dist, "cuda"))
    h2d = len(cells) * 40 + len(QS) * 8
    d2h = host_cut.nbytes

    # roofline of the sampler kernel (wide-multiply bound), from its CUDA-event
    # durations on the call's stream, summed over the waves of a step
    props = torch.cuda.get_device_properties(local)
    peaks = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz") or 2070.0)
    mul_peak = props.multi_processor_count * MUL_LANES_PER_SM * sm_max * 1e6 / 1e9  # Gmul/s
    kmean = statistics.mean(kern_ms)
    achieved = MUL_PER_DRAW * draws / (kmean / 1000.0) / 1e9
    h = kernel_source_hash()
    roofline = {"bound": "alu", "achieved": achieved, "peak": mul_peak, "unit": "Gmul/s (32x32->64)",
                "frac": achieved / mul_peak,
                "traffic": (TRAFFIC_PER_REPLICATE[h] * total_R / max(1, slaunch)
                            if h in TRAFFIC_PER_REPLICATE and args.workload == "sweep" else None),
                "kernel": ("mn_sample_kernel" if args.sampler == "multinomial"
                           else "sample_block_kernel" if args.workload == "large-n"
                           else "sample_hist_kernel + sample_block_kernel" if args.workload == "batched"
                           else "sample_hist_kernel"),
                "kernel_ms_per_step": kmean, "launches_per_step": slaunch,
                "finisher_ms_per_step": statistics.mean(fin_ms),
                "peak_basis": f"{props.multi_processor_count} SMs x {MUL_LANES_PER_SM} multiply lanes x "
                              f"{sm_max:.0f} MHz (max SM clock of MEASURED_PEAKS.json); "
                              f"{MUL_PER_DRAW} multiplies per draw"}

    line = {"metric": METRIC, "value": value, "unit": "replicates/s", "samples_per_s": sps,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64" if prec == pl.PL_FP32_BULK else "f64",
            "data": "synthetic (Philox streams, seed 1)", "config": config,
            "e2e": {"value": e2e_value, "unit": "replicates/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "roofline": roofline, "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_oracle_rate(args.cpu_sample, threads)
        line["cpu_baseline"] = {"value": cb["value"], "unit": "replicates/s", "cores": threads,
                                "kind": "oracle", "sample": cb["sample"],
                                "samples_per_s": cb["samples_per_s"]}
        if args.workload == "sweep":  # the same oracle on one core, a smaller sample
            c1 = cpu_oracle_rate(max(1, args.cpu_sample // 8), 1)
            line["cpu_baseline"]["one_core"] = {"value": c1["value"], "cores": 1, "sample": c1["sample"]}
    main_sweep = args.workload == "sweep" and world == 1 and args.sampler == "inverse-cdf"
    f64_flops = None
    if main_sweep and not args.no_extras:
        probe = ctx.pl_probe_rates()
        line["probe"] = probe
        roofline["probe"] = {k: probe[k] for k in ("sm_clock_mhz", "mul_wide_per_sm_clk", "philox_words_per_s")}
        f64_peak = props.multi_processor_count * probe["dfma_per_sm_clk"] * sm_max * 1e6 / 1e9  # Gflop/s of FMA
        f64_flops = 2.0 * f64_peak
        roofline["finisher"] = finisher_roofline(statistics.mean(fin_ms), total_R, waves, f64_peak, probe)
        line["fp64_form"] = fp64_form_record(ctx, cells, seed, QS, flush, torch, stream, pl, value)
        line["c0_fp64"] = c0_fp64_record(ctx, flush, torch, stream, pl)
    if main_sweep and not args.no_per_cell:
        line["per_cell"] = per_cell_rates(ctx, cells, seed, QS, prec, mul_peak, flush, torch,
                                          f64_peak_gflops=f64_flops)
    if main_sweep and not args.no_extras:
        ctx.close()
        ctx = None
        m = serve_measure(local, args.extras_serve_s, 3.0, args.workers, pl.PL_FP32_BULK, pl, torch)
        line["serving"] = {"workload": serving_config(args)["workload"], "offered_per_s": SERVE_RATE,
                           "value": m["value"], "unit": "requests/s", "measured_s": args.extras_serve_s,
                           "warmup_s": 3.0, "requests": len(m["timed"]), "latency_ms": m["latency_ms"],
                           "failed_requests": m["failed_requests"], "draws_per_s": m["draws_per_s"],
                           "load": m["load"], "clocks": m["clocks"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ctx is not None:
        ctx.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
