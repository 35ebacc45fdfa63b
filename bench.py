"""Benchmark: checked accesses per second on the global-memory workload.

Workload (one step = one full check of one trace): a grid of 1024 blocks x 256
threads over 2^26 shadowed words, 256 accesses per thread (70% read, 25% write,
5% atomicAdd; half block-strided in the block's own tile, half uniform-random),
__syncwarp every 8 and __syncthreads every 32 accesses, 0.1% of the words made
racy across blocks: 67,108,864 accesses + 8,126,464 barrier records
(75,235,328 records, 1.20 GB).  Synthetic, seeded; inputs (1.2 GB trace,
512 MB shadow) are larger than L2, so no flush is needed between steps.

Each timed step checks the trace as the next kernel launch of the same region
(kernel_base = step), so the shadow's kernel tags make older values read as
INIT and every eighth step includes the group clear of the whole shadow.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

N > 1 runs under torch.distributed.run: every rank checks its own replica of
the workload (the checker shards by independent trace, no collective on the
data path); value = all ranks' accesses / max-over-ranks time.
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
sys.path.insert(0, ROOT)

METRIC = "checked accesses/sec vs HBM roofline"
UNIT = "accesses/s"
WORKLOAD = "global-mix: 1024x256 threads, 2^26 words, 67.1M accesses + 8.1M barrier records"


def workload_name(n_blocks, n_words, n_acc, n_sync):
    """Label of the global-mix workload actually run (the default is WORKLOAD)."""
    if n_blocks == 1024:
        return WORKLOAD
    return "global-mix: %dx256 threads, %d words, %.1fM accesses + %.1fM barrier records" % (
        n_blocks, n_words, n_acc / 1e6, n_sync / 1e6)
ALG_BYTES_PER_ACCESS = 32   # 16 B record + 8 B shadow read + 8 B shadow write
ALG_BYTES_PER_SYNC = 16     # a barrier record is streamed, not an access
ALG_BYTES_PER_ACCESS_COMPACT = 24  # 16 B record + 4 B shadow read + 4 B shadow write


KERNEL_SOURCES = ("paper_2401_04701_gb300/csrc/hr_kernels.cu", "paper_2401_04701_gb300/csrc/hr_binned.cu",
                  "paper_2401_04701_gb300/csrc/hr_internal.h", "include/hirace_device.cuh")
BINNED_KERNELS = "hr_bin_count, hr_bin_scan_sums, hr_bin_scan, hr_bin_scatter, hr_bin_groups"


def kernel_sources_sha():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(variant):
    """DRAM bytes of one check (the kernels after the pre-pass) with this checker
    variant, from the committed ncu capture; None when the kernel sources changed
    since it was taken or the variant was not captured."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        e = t.get("checks", {}).get(str(variant))
        if e and t.get("kernel_sources_sha256") == kernel_sources_sha():
            return int(e["dram_bytes_read"]) + int(e["dram_bytes_write"])
    except Exception:
        pass
    return None


def checker_name(variant):
    """The kernels one check runs after the pre-pass, for the JSON line."""
    from paper_2401_04701_gb300 import hirace
    if dict(hirace.variants())[variant]["binned"]:
        return "binned checker (variant %d): %s" % (variant, BINNED_KERNELS)
    return "hr_check_kernel variant %d" % variant


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(gpu_index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.15)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(value, device=None):
    """The largest per-rank value (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([float(value)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank_per_step, steps, max_ms):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank_per_step * steps / (max_ms / 1e3)


def make_workload(n_blocks=1024, kind="global", log2_vertices=22):
    """The benchmark workload (global mix, `n_blocks` x 256 threads), or with
    --workload the power-law push (2^log2_vertices vertices, 4 sweeps) or the
    tree reduction: (trace, info, accesses, barrier records)."""
    from paper_2401_04701_gb300 import tracegen as tg
    if kind == "powerlaw":
        trace, info = tg.gen_powerlaw_push(tg.seed_for(3), log2_vertices=log2_vertices)
    elif kind == "tree":
        trace, info = tg.gen_tree_reduction(tg.seed_for(1), inject=True)
    else:
        trace, info = tg.gen_global_mix(tg.seed_for(2), inject=True, n_blocks=n_blocks)
    n_acc = int(np.count_nonzero(trace["op"] <= tg.OP_A))
    n_sync = len(trace) - n_acc
    return trace, info, n_acc, n_sync


def host_cores():
    return len(os.sched_getaffinity(0))


def cpu_oracle_rate(trace, info, n_acc, max_records=None, threads=1):
    """Serial FSM oracle (C) over a sample of the trace, on one core or on
    `threads` cores (disjoint word ranges): (accesses/s, seconds, accesses)."""
    from oracle import oracle
    sample = trace if max_records is None else trace[:max_records]
    acc = int(np.count_nonzero(sample["op"] <= 2)) if max_records is not None else n_acc
    t0 = time.perf_counter()
    if threads > 1:
        oracle.serial_fsm_parallel(sample, info["block_dim"], info["n_words"], threads=threads)
    else:
        oracle.serial_fsm(sample, info["block_dim"], info["n_words"])
    dt = time.perf_counter() - t0
    return acc / dt, dt, acc


def instrumented_slowdown(dev, reps=20):
    """Time each synthetic kernel without and with inline hr_access() calls
    (1,048,576 threads, block 256; clean variants).  Returns per-kernel ms and
    the slowdown ratio; the instrumented runs check a fresh kernel each rep."""
    import torch
    from paper_2401_04701_gb300 import hirace
    hirace.load_workloads()
    n, n_bins = 1 << 20, 4096
    d_in = torch.rand(n, device=dev)
    d_out = torch.zeros(n, device=dev)
    keys = torch.randint(0, n_bins, (n,), device=dev, dtype=torch.int32)
    bins = torch.zeros(n_bins, dtype=torch.int32, device=dev)
    red = torch.rand(n, device=dev)
    sums = torch.zeros(n // 256, device=dev)
    jobs = {
        "stencil": (2 * n, lambda v: hirace.run_stencil(v, d_in, d_out)),
        "histogram": (n_bins, lambda v: hirace.run_histogram(v, keys, bins)),
        "reduction": (n, lambda v: hirace.run_reduce(v, red)),
        # block reduction in __shared__ memory, its shadow in HBM or beside it in shared memory
        "shared_reduction_hbm_shadow": (n, lambda v: hirace.run_smem_reduce(v, d_in, sums, 0 if v is None else 1)),
        "shared_reduction_smem_shadow": (n, lambda v: hirace.run_smem_reduce(v, d_in, sums, 0 if v is None else 2)),
    }
    out = {}
    stream = torch.cuda.current_stream(dev)
    for name, (n_words, fn) in jobs.items():
        with hirace.Checker([dict(n_words=n_words, block_dim=256)], report_capacity=1 << 16) as ck:
            times = {}
            for mode in ("plain", "instrumented"):
                total = 0.0
                for r in range(reps + 2):
                    view = ck.device_view(0) if mode == "instrumented" else None
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    a.record(stream)
                    fn(view)
                    b.record(stream)
                    torch.cuda.synchronize()
                    if r >= 2:
                        total += a.elapsed_time(b)
                    if mode == "instrumented":
                        ck.sync(0)
                times[mode] = total / reps
            _, status, n_total, _ = ck.report(0)
        out[name] = {"plain_ms": times["plain"], "instrumented_ms": times["instrumented"],
                     "slowdown": times["instrumented"] / times["plain"], "races": n_total,
                     "status": hirace.STATUS[status]}
    gm = float(np.exp(np.mean([np.log(v["slowdown"]) for v in out.values()])))
    return {"kernels": out, "slowdown_geomean": gm, "threads": n, "block": 256}


def other_workloads(dev, reps=5):
    """The tree-reduction workload (1 block, 1,029,952+ records) and the power-law
    push workload (2^22 vertices, 4 sweeps, 536,870,912 records): the autotuner's
    times, and accesses/s of the warp-aggregated and the plain kernel of one shape
    (2 records per lane, 8 consumer warps), FSM-kernel time from the library's events."""
    import torch
    from paper_2401_04701_gb300 import hirace, tracegen as tg
    out = {}
    cases = [("tree_reduction_shared_1x256", lambda: tg.gen_tree_reduction(tg.seed_for(1), inject=True)),
             ("powerlaw_push_2^22v_16deg_4sweeps", lambda: tg.gen_powerlaw_push(tg.seed_for(3)))]
    for name, make in cases:
        trace, info = make()
        n_acc = int(np.count_nonzero(trace["op"] <= 2))
        d = torch.from_numpy(trace.view(np.uint8)).to(dev)
        res = {"records": len(trace), "accesses": n_acc}
        with hirace.Checker([dict(n_words=info["n_words"], block_dim=info["block_dim"])],
                            report_capacity=1 << 22) as ck:
            best, tune_ms = ck.autotune(0, d)
            res["autotuned"] = {"variant": best, "desc": dict(hirace.variants())[best],
                                "kernel_ms": tune_ms[best], "accesses_per_s": n_acc / (tune_ms[best] / 1e3),
                                "ms_per_variant": [round(t, 4) for t in tune_ms]}
            ck.set_variant(2)  # the 2-records-per-lane, 8-consumer shape: aggregated (2) against plain (3)
            for agg in (True, False):
                ck.reset(0)
                ck.check_trace(0, d, aggregate=agg)
                ck.report(0)
                ck.profile(True)
                ck.profile_read()
                start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                tot = 0.0
                for _ in range(reps):
                    ck.reset(0)
                    torch.cuda.synchronize()
                    start.record()
                    ck.check_trace(0, d, aggregate=agg)
                    stop.record()
                    torch.cuda.synchronize()
                    tot += start.elapsed_time(stop)
                prof = ck.profile_read()
                ck.profile(False)
                races, status, n_total, _ = ck.report(0)
                cnt = ck.counters(0)
                key = "aggregated" if agg else "plain"
                res[key] = {"accesses_per_s": n_acc * reps / (tot / 1e3), "ms_per_check": tot / reps,
                            "kernel_ms": prof["check_ms"] / max(1, prof["calls"]), "races": n_total,
                            "status": hirace.STATUS[status], "cas_last_check": int(cnt["cas"]),
                            "merged_lanes_last_check": int(cnt["merged"])}
        out[name] = res
        del d
        torch.cuda.empty_cache()
    return out


def compact_shadow_workload(dev, d_trace, info, n_acc, n_sync, variant, p_hbm, reps=10):
    """The same global-mix trace on a compact 4-byte shadow (18-bit tids, 3-bit
    bc and wc; 256 MB instead of 512 MB).  Its algorithmic bytes are 16 B of
    record + 4 B read + 4 B written per access."""
    import torch
    from paper_2401_04701_gb300 import hirace
    reg = dict(n_words=info["n_words"], block_dim=info["block_dim"], shadow_bytes=4, tid_bits=18)
    with hirace.Checker([reg], report_capacity=1 << 22) as ck:
        ck.set_variant(variant)
        ck.check_trace(0, d_trace)
        races, status, n_total, _ = ck.report(0)
        ok = status == hirace.HR_OK and n_total == len(info["injected"])
        for kb in range(1, 4):
            ck.check_trace(0, d_trace, kernel_base=kb)
        torch.cuda.synchronize()
        ck.profile(True)
        ck.profile_read()
        for kb in range(4, 4 + reps):
            ck.check_trace(0, d_trace, kernel_base=kb)
        torch.cuda.synchronize()
        prof = ck.profile_read()
        ck.profile(False)
        _, status, _, _ = ck.report(0)
    check_ms = prof["check_ms"] / max(1, prof["calls"])
    alg = n_acc * ALG_BYTES_PER_ACCESS_COMPACT + n_sync * ALG_BYTES_PER_SYNC
    return {"shadow_bytes_per_word": 4, "tid_bits": 18, "races_match": bool(ok), "status": hirace.STATUS[status],
            "kernel_ms": check_ms, "accesses_per_s": n_acc / (check_ms / 1e3),
            "alg_bytes_per_launch": alg, "frac_of_hbm_roofline": alg / (check_ms / 1e3) / 1e9 / p_hbm}


def every_epoch_workload(dev, d_trace, info, n_acc, n_sync, p_hbm, reps=10):
    """The same global-mix trace with every racy epoch reported (RACE not
    absorbing; per-conflict-bit summaries, 24 shadow bytes per word)."""
    import torch
    from paper_2401_04701_gb300 import hirace
    reg = dict(n_words=info["n_words"], block_dim=info["block_dim"], report_mode=hirace.REPORT_EVERY_EPOCH)
    with hirace.Checker([reg], report_capacity=1 << 22) as ck:
        ck.check_trace(0, d_trace)
        races, status, n_reports, _ = ck.report(0)
        ok = status == hirace.HR_OK and set(races["word"].tolist()) == set(info["injected"].tolist())
        for kb in range(1, 4):
            ck.check_trace(0, d_trace, kernel_base=kb)
        torch.cuda.synchronize()
        ck.profile(True)
        ck.profile_read()
        for kb in range(4, 4 + reps):
            ck.check_trace(0, d_trace, kernel_base=kb)
        torch.cuda.synchronize()
        prof = ck.profile_read()
        ck.profile(False)
        _, status, _, _ = ck.report(0)
    check_ms = prof["check_ms"] / max(1, prof["calls"])
    alg = n_acc * ALG_BYTES_PER_ACCESS + n_sync * ALG_BYTES_PER_SYNC
    return {"shadow_bytes_per_word": 24, "reports_per_check": int(n_reports), "racy_words_match": bool(ok),
            "status": hirace.STATUS[status], "kernel_ms": check_ms, "accesses_per_s": n_acc / (check_ms / 1e3),
            "frac_of_hbm_roofline_at_32B_per_access": alg / (check_ms / 1e3) / 1e9 / p_hbm}


def batch_workload(dev, reps=3):
    """512 traces (lengths log-uniform 10K..10M records, 60% shared-memory, 40%
    global-memory) checked three ways: one launch per trace, one batched launch,
    and the batched launch replayed from a CUDA graph, all with the per-wave shape
    whose batched launch was fastest.  Resets run outside the timed spans."""
    import torch
    from paper_2401_04701_gb300 import hirace, tracegen as tg
    jobs = tg.gen_batch(tg.seed_for(4))
    n_acc = sum(int(np.count_nonzero(tr["op"] <= 2)) for tr, _ in jobs)
    n_rec = sum(len(tr) for tr, _ in jobs)
    regions = [dict(n_words=info["n_words"], block_dim=info["block_dim"], report_capacity=1 << 14)
               for _, info in jobs]
    d = [torch.from_numpy(tr.view(np.uint8)).to(dev) for tr, _ in jobs]
    del jobs
    out = {"traces": len(d), "records": n_rec, "accesses": n_acc}
    stream = torch.cuda.current_stream(dev)
    with hirace.Checker(regions, report_capacity=1 << 14) as ck:
        ck.batch_reserve(len(d), 1 << 18)

        def reset_all():
            for i in range(len(d)):
                ck.reset(i)
            torch.cuda.synchronize()

        def timed(fn):
            tot = 0.0
            for r in range(reps + 1):
                reset_all()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                torch.cuda.synchronize()
                if r:
                    tot += a.elapsed_time(b)
            return tot / reps

        # the per-wave shape for this batch: one timed batched launch per shape, the fastest kept
        shape_ms = []
        for v in range(6):
            ck.set_variant(v)
            reset_all()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ck.check_batch(list(enumerate(d)))
            b.record(stream)
            torch.cuda.synchronize()
            shape_ms.append(a.elapsed_time(b))
        ck.set_variant(int(np.argmin(shape_ms)))
        out["variant"] = int(np.argmin(shape_ms))
        out["batched_ms_per_variant"] = [round(t, 3) for t in shape_ms]
        per_trace_ms = timed(lambda: [ck.check_trace(i, t) for i, t in enumerate(d)])
        races_single = sum(ck.report(i)[2] for i in range(len(d)))
        # per-trace completion times: one launch per trace (events after each launch)
        reset_all()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(d) + 1)]
        evs[0].record(stream)
        for i, t in enumerate(d):
            ck.check_trace(i, t)
            evs[i + 1].record(stream)
        torch.cuda.synchronize()
        done_single = np.array([evs[0].elapsed_time(e) for e in evs[1:]])
        batch_ms = timed(lambda: ck.check_batch(list(enumerate(d))))
        races_batch = sum(ck.report(i)[2] for i in range(len(d)))
        done_batch = ck.batch_job_times(len(d)) / 1e6   # the last timed batch, device clock
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(dev)
        reset_all()
        with torch.cuda.stream(s):
            ck.check_batch(list(enumerate(d)), stream=s)
        torch.cuda.synchronize()
        reset_all()
        with torch.cuda.graph(g, stream=s):
            ck.check_batch(list(enumerate(d)), stream=s)
        graph_ms = timed(lambda: g.replay())
        races_graph = sum(ck.report(i)[2] for i in range(len(d)))
    for name, ms in (("one_launch_per_trace", per_trace_ms), ("batched_launch", batch_ms),
                     ("batched_graph_replay", graph_ms)):
        out[name] = {"ms": ms, "accesses_per_s": n_acc / (ms / 1e3)}
    out["races"] = {"per_trace": races_single, "batched": races_batch, "graph": races_graph}
    for name, done in (("one_launch_per_trace", done_single), ("batched_launch", done_batch)):
        out[name]["trace_completion_ms"] = {"p50": float(np.percentile(done, 50)),
                                            "p99": float(np.percentile(done, 99)), "max": float(done.max())}
    return out


def serving_workload(dev, duration, rates=(2000.0,), serial_duration=None):
    """The serving measurement at the workload's 2000 requests/s (and, with
    --all-workloads, at a higher rate where one-at-a-time service saturates)."""
    from paper_2401_04701_gb300 import serving
    pool = serving.TracePool(dev, scale="full")
    return {"%d_per_s" % r: serving_run(dev, pool, duration, r, serial_duration) for r in rates}


def serving_run(dev, pool, duration, rate, serial_duration=None):
    """Poisson arrivals (rate/s for `duration` s): 75% trace checks (prefixes of
    10K..50M records of pooled tree-reduction, global-mix and power-law traces),
    25% instrumented kernels (grid 64..4096 x 256, on streams of their own); 64
    region slots, 64 GB shadow budget, 64M records per iteration shared by the
    active jobs (at least 1M each).  Then the same arrivals (the first
    `serial_duration` seconds of them, default all) served one request at a
    time (whole trace per check) for at most twice as long."""
    from paper_2401_04701_gb300 import serving
    reqs = serving.make_requests(tg_seed(5), rate=rate, duration=duration)
    srv = serving.Server(pool, dev, n_slots=64, slot_words=1 << 26, budget_bytes=64 << 30, chunk_records=1 << 20)
    t0 = time.perf_counter()
    res = srv.run(reqs)
    wall = time.perf_counter() - t0
    out = {"requests": len(reqs), "rate_per_s": rate, "duration_s": duration,
           "continuous_batching": dict(serving.summarize(res, wall), iterations=srv.iterations, wall_s=wall,
                                       overlapped_launches=srv.overlapped)}
    sd = duration if serial_duration is None else min(duration, serial_duration)
    sreqs = [r for r in reqs if r.arrival <= sd]
    ser = serving.Server(pool, dev, n_slots=2, slot_words=1 << 26, budget_bytes=64 << 30)
    t0 = time.perf_counter()
    sres = ser.run_serial(sreqs, time_limit=2 * sd)
    swall = time.perf_counter() - t0
    out["serial_one_at_a_time"] = dict(serving.summarize(sres, swall), wall_s=swall, requests=len(sreqs),
                                       arrivals_s=sd, not_served=len(sreqs) - len(sres))
    return out


def tg_seed(k):
    from paper_2401_04701_gb300 import tracegen as tg
    return tg.seed_for(k)


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle as it stands, on the host cores, over the
    whole benchmark trace each step (the same workload the GPU arm checks)."""
    if rank != 0:
        return
    trace, info, n_acc, n_sync = make_workload()
    cores = host_cores()
    for _ in range(args.warmup):
        cpu_oracle_rate(trace, info, n_acc, threads=cores)
    tot_acc, tot_t = 0, 0.0
    for _ in range(args.steps):
        _, dt, acc = cpu_oracle_rate(trace, info, n_acc, threads=cores)
        tot_acc += acc
        tot_t += dt
    value = tot_acc / tot_t
    sample = ("the whole workload each step (%d records, %d accesses): serial FSM oracle in C on %d disjoint word "
              "ranges, one host thread each" % (len(trace), n_acc, cores))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "whole trace"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def check_latency(ck, d_trace, stream, expect, n):
    """Latency of one check issued alone: n times, reset the region, then
    hr_check_trace on an idle stream (device time between CUDA events around
    it) and hr_report (host time from the check's submission until the race
    records are on the host).  Runs after the throughput loop, outside its
    timed region.  p50 / p99 / max in ms."""
    import torch
    from paper_2401_04701_gb300 import hirace
    if n <= 0:
        return None
    dev_ms, rep_ms = [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(n):
        ck.reset(0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0.record(stream)
        ck.check_trace(0, d_trace)
        e1.record(stream)
        _, status, n_total, _ = ck.report(0)
        rep_ms.append((time.perf_counter() - t0) * 1e3)
        dev_ms.append(e0.elapsed_time(e1))
        if status != hirace.HR_OK or n_total != expect:
            raise SystemExit("latency check failed: status %s, %d races" % (hirace.STATUS[status], n_total))

    def q(v):
        v = np.asarray(v)
        return {"p50": float(np.percentile(v, 50)), "p99": float(np.percentile(v, 99)), "max": float(v.max())}
    return {"checks": n, "device_ms": q(dev_ms), "to_report_ms": q(rep_ms),
            "what": "one check of the whole trace issued alone after a reset: device time of hr_check_trace, "
                    "and host time from its submission until hr_report returned the race records"}


def run_gpu(args, rank, world, local_rank):
    import torch
    from paper_2401_04701_gb300 import hirace

    dist = None
    if world > 1:
        import torch.distributed as dist
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    hirace.load_library()

    trace, info, n_acc, n_sync = make_workload(args.blocks, args.workload, args.log2_vertices)
    default = args.workload == "global" and args.blocks == 1024
    host = torch.from_numpy(trace.view(np.uint8)).pin_memory()
    d_trace = host.to(dev)
    stream = torch.cuda.current_stream(dev)
    ring = 1 << 22
    ck = hirace.Checker([dict(n_words=info["n_words"], block_dim=info["block_dim"])], report_capacity=ring)

    # the autotuner picks the kernel variant (tile shape, aggregation) on this workload,
    # unless --variant pins one (profiling runs, where tuning under a profiler misleads)
    if args.variant is None:
        best, tune_ms = ck.autotune(0, d_trace)
    else:
        ck.set_variant(args.variant)
        best, tune_ms = args.variant, None
    # correctness gate: one check vs the injected set (the global mix's racy words
    # are exactly its injected words; the other workloads' parity is in the tests,
    # here later checks must repeat the first one's count)
    ck.check_trace(0, d_trace)
    races, status, n_total, _ = ck.report(0)
    gate_races = races
    expect = len(info["injected"]) if args.workload == "global" else n_total
    if status != hirace.HR_OK or n_total != expect:
        raise SystemExit("bench workload check failed: status %s, %d races" % (hirace.STATUS[status], n_total))
    ck.reset(0)
    torch.cuda.synchronize()

    # every check is a later launch: kernel ordinals advance by the trace's kernel count
    kstep = int(trace["kernel"].max()) + 1 if len(trace) else 1
    kb = 0
    for _ in range(args.warmup):
        ck.check_trace(0, d_trace, kernel_base=kb)
        kb += kstep
    torch.cuda.synchronize()
    ck.profile(True)
    ck.profile_read()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank) if rank == 0 else None
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for _ in range(args.steps):
        ck.check_trace(0, d_trace, kernel_base=kb)
        kb += kstep
    stop.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop() if clocks else None
    ms = start.elapsed_time(stop)
    prof = ck.profile_read()
    ck.profile(False)
    counters = ck.counters(0)
    _, status, _, _ = ck.report(0)
    if status != hirace.HR_OK:
        raise SystemExit("timed steps ended with %s" % hirace.STATUS[status])
    ms = max_over_ranks(ms, dev)

    # end to end through the C-ABI from pinned host memory: reset, the check of
    # the host trace (hr_check_trace_host: its H2D copies overlap the checks of
    # the chunks before them), D2H of the race records
    e2e_steps = 0 if args.no_e2e else max(1, min(args.steps, 10))
    d2h = 0
    ck.reset(0)
    ck.check_trace_host(0, host)   # sizes the staging buffers outside the timed loop
    ck.report(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ck.reset(0)
        ck.check_trace_host(0, host)
        races, status, n_total, _ = ck.report(0)
        d2h += races.nbytes + 64
        if status != hirace.HR_OK or n_total != expect:
            raise SystemExit("end-to-end check failed: status %s, %d races" % (hirace.STATUS[status], n_total))
    e2e_s = time.perf_counter() - t0
    e2e_rate = world * n_acc * e2e_steps / e2e_s if e2e_steps else None
    # the host link's own ceiling beside it: plain pinned H2D copies of the same bytes
    h2d_gbs = None
    if e2e_steps:
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        d_trace.copy_(host, non_blocking=True)
        c0.record()
        for _ in range(3):
            d_trace.copy_(host, non_blocking=True)
        c1.record()
        torch.cuda.synchronize()
        h2d_gbs = 3 * host.numel() / (c0.elapsed_time(c1) / 1e3) / 1e9
    latency = check_latency(ck, d_trace, stream, expect, args.latency_checks) if default else None

    if rank != 0:
        ck.close()
        return
    value = job_rate(world, n_acc, args.steps, ms)
    p_hbm, peak_kind = peaks()
    alg_bytes = n_acc * ALG_BYTES_PER_ACCESS + n_sync * ALG_BYTES_PER_SYNC
    check_ms = prof["check_ms"] / max(1, prof["calls"])
    achieved = alg_bytes / (check_ms / 1e3) / 1e9
    cpu = None
    if not args.no_cpu_baseline and default:
        cores = host_cores()
        rate, dt, acc = cpu_oracle_rate(trace, info, n_acc, threads=cores)
        rate1, dt1, _ = cpu_oracle_rate(trace, info, n_acc)
        from oracle import oracle
        t0 = time.perf_counter()
        bf = oracle.bruteforce_parallel(trace, info["block_dim"], info["n_words"], threads=cores)
        dtb = time.perf_counter() - t0
        # the GPU's racy (kernel, word, epoch) set of the correctness-gate check
        # against the brute force on the same trace
        match = hirace.race_keys(gate_races) == oracle.race_keys(bf)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "whole workload once (%d accesses, %.1f s): serial FSM oracle in C on %d disjoint "
                         "word ranges, one host thread each" % (acc, dt, cores),
               "single_core": {"value": rate1, "cores": 1, "seconds": dt1},
               "bruteforce_all_cores": {"value": n_acc / dtb, "cores": cores, "seconds": dtb,
                                        "racy_words": int(len(bf)), "racy_words_match": bool(match)}}
        if not match:
            raise SystemExit("GPU race set differs from the oracle's brute force on the benchmark trace")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": workload_name(args.blocks, info["n_words"], n_acc, n_sync) if args.workload == "global"
                   else "%s: %d records, %d words" % (args.workload, len(trace), info["n_words"]),
                   "n_words": info["n_words"], "records": len(trace), "accesses": n_acc,
                   "shadow_bytes_per_word": 8, "racy_words": int(expect),
                   "l2": "inputs larger than L2 (%.2f GB trace, %d MB shadow), no flush" % (
                       len(trace) * 16 / 1e9, info["n_words"] * 8 >> 20),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": p_hbm, "unit": "GB/s",
                     "frac": achieved / p_hbm, "traffic": measured_traffic(best) if default else None,
                     "kernel": checker_name(best),
                     "peak_kind": peak_kind, "alg_bytes_per_launch": alg_bytes,
                     "kernel_ms": check_ms, "prepass_ms": prof["prepass_ms"] / max(1, prof["calls"])},
        "e2e": {"value": e2e_rate, "unit": UNIT, "h2d_bytes_per_step": int(host.numel()),
                "d2h_bytes_per_step": int(d2h // max(1, e2e_steps)),
                "h2d_gbs_in_checks": host.numel() * e2e_steps / e2e_s / 1e9 if e2e_steps else None,
                "pinned_h2d_copy_gbs": h2d_gbs},
        "fsm_counters": {k: int(v) for k, v in counters.items()},
        "gpu_launches": int(prof["launches"]),
        "autotune": {"chosen": best, "variant": dict(hirace.variants())[best],
                     "ms_per_variant": [round(t, 4) for t in tune_ms] if tune_ms else "pinned by --variant"},
        "clocks": clk,
    }
    if latency:
        line["check_latency"] = latency
    if cpu:
        line["cpu_baseline"] = cpu
    if default and not args.no_mode_lines:
        line["compact_shadow"] = compact_shadow_workload(dev, d_trace, info, n_acc, n_sync, best, p_hbm)
        line["every_epoch_reports"] = every_epoch_workload(dev, d_trace, info, n_acc, n_sync, p_hbm)
    if not args.no_instrumented:
        line["instrumented_slowdown"] = instrumented_slowdown(dev)
    if not args.quick:
        # the other workloads: tree reduction and power-law push (per-wave and
        # autotuned, plain vs warp-aggregated), the 512-trace batch (one launch
        # per trace vs one batched launch vs CUDA-graph replay), and serving at
        # 2000 requests/s (continuous batching vs one request at a time)
        t0 = time.perf_counter()
        line["other_workloads"] = other_workloads(dev)
        line["batch_workload"] = batch_workload(dev)
        rates = (2000.0, 8000.0) if args.all_workloads else (2000.0,)
        line["serving"] = serving_workload(dev, args.serving_seconds, rates, args.serial_seconds)
        line["other_workloads_wall_s"] = time.perf_counter() - t0
    print(json.dumps(line), flush=True)
    ck.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-instrumented", action="store_true")
    ap.add_argument("--quick", action="store_true",
                    help="only the global-mix line (no tree, power-law, batch or serving runs)")
    ap.add_argument("--all-workloads", action="store_true",
                    help="also serve 8000 requests/s (over capacity for one-at-a-time service)")
    ap.add_argument("--serving-only", action="store_true", help="run only the serving measurement")
    ap.add_argument("--serving-seconds", type=float, default=60.0,
                    help="length of the Poisson arrival run (the serving workload is 60 s)")
    ap.add_argument("--serial-seconds", type=float, default=60.0,
                    help="arrivals the one-request-at-a-time baseline serves (the first this many seconds)")
    ap.add_argument("--latency-checks", type=int, default=50,
                    help="single checks timed one at a time for the p50/p99 check latency (default workload)")
    ap.add_argument("--variant", type=int, default=None,
                    help="pin the checker kernel variant instead of autotuning")
    ap.add_argument("--no-mode-lines", action="store_true",
                    help="skip the compact-shadow and every-epoch lines (profiling runs)")
    ap.add_argument("--workload", default="global", choices=["global", "powerlaw", "tree"],
                    help="time another workload instead of the global mix (parity is in the tests)")
    ap.add_argument("--log2-vertices", type=int, default=22, help="power-law workload size")
    ap.add_argument("--blocks", type=int, default=1024,
                    help="scale the workload (profiling only; the benchmark is 1024)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.serving_only:
        import torch
        torch.cuda.set_device(local_rank)
        print(json.dumps({"serving": serving_workload(torch.device("cuda", local_rank), args.serving_seconds)}))
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    run_gpu(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
