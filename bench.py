#!/usr/bin/env python3
"""Benchmark of the GB300 access-mode consistency checker.

Headline step = one amc_check_trace call over the 2^30-op, 2^20-variable
Zipf(1.05) trace (kind mix r .40 / w .20 / Push .15 / Pull .15 / Noop .10, fair
side, seed 1): every per-step status, final status and first fault.  Inputs
(5.4 GB) are resident in HBM when the timed region starts and exceed L2, so no
L2 flush is needed between steps.

The same JSON line carries, under "configs", the other workloads, each timed
with CUDA events on its own stream with its clocks sampled and its oracle
timed on the host cores beside it:
  uniform_4096  16 variables, 4,096 uniform ops (seed 0): latency per check;
  vectorpu      2^24 VectorPU calls over 4,096 overlapping arrays (seed 2):
                translation + guarded check per step;
  vectorpu_lifetimes  2^24 VectorPU calls over 16 vectors and 65,536
                pvectors created and deleted during the run (seed 6):
                translation with live overlap sets + check with inherited
                statuses per step;
  trace_sizes   the trace check on Zipf traces of 2^24, 2^26 and 2^28 ops
                and on a 2^30-op low-fault trace;
  programs      100,000 If/While programs (seed 3): the batched persistent
                launch (CUDA graph) against one launch per program;
  programs_guarded  20,000 programs whose If conditions test a guard
                variable (seed 7): the path-sensitive relation mode;
  serve         open-loop Poisson arrivals at 1k / 10k / 100k requests/s,
                half traces and half programs, latency from the scheduled
                arrival to the poll that sees the result.

Prints one JSON line (rank 0).  Under torchrun (N > 1) each rank checks its own
replica of the trace on its own GPU ("replicas only": the path has no exchange
step); value = ops of all ranks / max time over ranks; the sub-records run at
N = 1 only.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload all|trace|uniform|vectorpu|vectorpu_lifetimes|trace_sizes|
                              programs|well_declared|kloc|serve]
                  [--n-ops N] [--n-vars V] [--no-e2e] [--no-cpu]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PLAIN_STREAMS = 32      # concurrent streams of the per-program launches
METRIC = "checked ops/s + HBM GB/s vs peak, batched vs plain, bit-exact; serve p99 ms"
UNIT = "checked ops/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-ops", type=int, default=1 << 30)
    ap.add_argument("--n-vars", type=int, default=1 << 20)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-chunk", type=int, default=0, help="ops per chunk of the host-buffer check (0: 2^25)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--workload", default="all",
                    choices=["all", "trace", "uniform", "programs", "programs_guarded", "vectorpu",
                             "vectorpu_lifetimes", "trace_sizes", "well_declared", "kloc", "serve"])
    ap.add_argument("--rates", default="1000,10000,100000")
    ap.add_argument("--serve-requests", type=int, default=10_000)
    ap.add_argument("--serve-seconds", type=float, default=12.0, help="submission window per rate")
    ap.add_argument("--serve-drain-seconds", type=float, default=20.0, help="wait for results after submitting")
    ap.add_argument("--n-progs", type=int, default=100_000, help="programs workload: number of programs")
    ap.add_argument("--plain-progs", type=int, default=2000,
                    help="programs workload: programs timed with one launch each (0: none)")
    ap.add_argument("--sub-steps", type=int, default=10, help="timed steps of each sub-record")
    ap.add_argument("--sub-cpu-seconds", type=float, default=6.0)
    ap.add_argument("--threads", type=int, default=0, help="host threads of the all-cores baseline (0: all)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # raw samples: AMC_CLOCKS_DIR if set, else the temporary directory
        out_dir = os.environ.get("AMC_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"amc_clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device="cuda"):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate(ms_local, ops_local, world, device="cuda"):
    """Whole-job throughput: ops of all ranks over the slowest rank's time.
    Returns (ops_per_s, max_ms, total_ops)."""
    import torch
    ms = max_over_ranks(ms_local, world, device)
    total = float(ops_local)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([total], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        total = float(t.item())
    return total / (ms * 1e-3), ms, total


def cpu_baseline(ks_host, var_host, n_vars, budget_s):
    """The oracle as it stands, single-threaded, on a prefix of the same trace
    sized to about budget_s seconds."""
    import numpy as np
    import oracle
    oracle.build()
    n = min(1 << 22, len(ks_host))
    t0 = time.perf_counter()
    oracle.check_trace(ks_host[:n], var_host[:n], n_vars)
    dt = time.perf_counter() - t0
    want = n * budget_s / max(dt, 1e-6)                 # ops that take about budget_s
    m = int(min(len(ks_host), max(n, want)))
    reps = max(1, int(round(want / m)))                 # whole passes when the trace is shorter
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle.check_trace(ks_host[:m], var_host[:m], n_vars)
    dt = time.perf_counter() - t0
    what = "the whole trace" if m == len(ks_host) else f"the first {m} ops of the same trace"
    return {"value": reps * m / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{what} ({m} ops), {reps} pass(es), single thread ({dt:.1f} s)"}


def cpu_baseline_all(ks_host, var_host, n_vars, budget_s, threads):
    """The oracle on `threads` host threads, each taking the variables
    v % threads == t over the same prefix of the trace (every thread reads
    every op), repeated for about budget_s seconds."""
    import oracle
    oracle.build()
    m = min(len(ks_host), 1 << 28)
    reps, dt = timed_calls(lambda: oracle.check_trace_sharded(ks_host[:m], var_host[:m], n_vars, threads), budget_s)
    return {"value": reps * m / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"the first {m} ops of the same trace, {reps} pass(es), sharded by variable id modulo "
                      f"{threads} over {threads} threads ({dt:.1f} s)"}


def run_reference(args):
    """--impl reference: the CPU oracle on bounded samples of the same workload."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    import oracle
    import torch
    import workloads
    oracle.build()
    # the trace is generated on the GPU when one is present (same bytes as ours)
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    sample = min(args.n_ops, 1 << 26)
    ks, var = workloads.trace_zipf(args.n_ops, args.n_vars, seed=args.seed, device=dev)
    ks_h, var_h = ks[:sample].cpu().numpy(), var[:sample].cpu().numpy()
    del ks, var
    for _ in range(args.warmup):
        oracle.check_trace(ks_h[: 1 << 16], var_h[: 1 << 16], args.n_vars)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.check_trace(ks_h, var_h, args.n_vars)
        times.append(time.perf_counter() - t0)
    t = statistics.mean(times)
    value = sample / t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "zipf_trace", "n_ops": args.n_ops, "n_vars": args.n_vars, "zipf_s": 1.05,
                       "seed": args.seed, "sample_ops_per_step": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"first {sample} ops of the trace per step, single thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    import paper_1910_11110_gb300 as amc
    import workloads

    world, rank, local = dist_setup()
    amc.build()
    L = amc.lib()
    dev = torch.device("cuda", torch.cuda.current_device())
    n_ops, n_vars = args.n_ops, args.n_vars
    ks, var = workloads.trace_zipf(n_ops, n_vars, seed=args.seed, device=dev)
    torch.cuda.synchronize()
    out = dict(step_status=torch.empty(n_ops, dtype=torch.uint8, device=dev),
               final_status=torch.empty(n_vars, dtype=torch.uint8, device=dev),
               var_first_fault=torch.empty(n_vars, dtype=torch.int32, device=dev),
               first_fault=torch.empty(1, dtype=torch.int64, device=dev))
    ws = torch.empty(amc.trace_workspace_bytes(n_ops, n_vars) + 256, dtype=torch.uint8, device=dev)
    ws = ws[(-ws.data_ptr()) % 256:]
    # a stream of its own: once the size class is tuned, the library replays
    # the check as a captured graph (the legacy default stream cannot be captured)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())

    def step():
        amc.check_trace(ks, var, n_vars, out=out, workspace=ws, stream=stream)

    for _ in range(max(3, args.warmup)):
        step()
    if amc.sync_status() != 0:
        raise RuntimeError("device error during warm-up")

    # kernel events for the dominant kernel (recorded by the library on its stream)
    k_start = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    k_stop = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for ev in k_start + k_stop:      # torch creates the CUDA event on first record
        ev.record(stream)
    s_start = torch.cuda.Event(enable_timing=True)
    s_stop = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.4)
    barrier(world)
    torch.cuda.synchronize()
    s_start.record(stream)
    for i in range(args.steps):
        L.amc_set_profile_events(ctypes_ptr(k_start[i]), ctypes_ptr(k_stop[i]))
        step()
    L.amc_set_profile_events(None, None)
    s_stop.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    if amc.sync_status() != 0:
        raise RuntimeError("device error during timed steps")
    ms_total = s_start.elapsed_time(s_stop)
    value, ms_step, _ = aggregate(ms_total / args.steps, n_ops, world)
    k_ms = statistics.mean(a.elapsed_time(b) for a, b in zip(k_start, k_stop))

    peak, peak_kind = peaks()
    alg_bytes = 6 * n_ops + 5 * n_vars
    achieved = alg_bytes / (k_ms * 1e-3) / 1e9
    traffic = scan_traffic(n_ops, n_vars)

    # end-to-end through the public API: pinned host inputs, H2D, check, D2H
    e2e = None
    if not args.no_e2e:
        ks_h = torch.empty(n_ops, dtype=torch.uint8, pin_memory=True)
        var_h = torch.empty(n_ops, dtype=torch.int32, pin_memory=True)
        ks_h.copy_(ks)
        var_h.copy_(var)
        hout = dict(step_status=torch.empty(n_ops, dtype=torch.uint8, pin_memory=True),
                    final_status=torch.empty(n_vars, dtype=torch.uint8, pin_memory=True),
                    var_first_fault=torch.empty(n_vars, dtype=torch.int32, pin_memory=True),
                    first_fault=torch.empty(1, dtype=torch.int64, pin_memory=True))
        hws = torch.empty(amc.trace_host_workspace_bytes(n_ops, n_vars, args.e2e_chunk) + 256, dtype=torch.uint8,
                          device=dev)
        hws = hws[(-hws.data_ptr()) % 256:]

        def e2e_step():
            # one call: chunked H2D of the pinned inputs, checks, D2H of every output
            amc.check_trace_host(ks_h, var_h, n_vars, chunk_ops=args.e2e_chunk, out=hout, workspace=hws,
                                 stream=stream)

        e2e_step()
        torch.cuda.synchronize()
        n_e2e = max(1, min(args.steps, 5))
        barrier(world)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n_e2e):
            e2e_step()
        b.record(stream)
        torch.cuda.synchronize()
        e_ms = max_over_ranks(a.elapsed_time(b) / n_e2e, world)
        e2e = {"value": n_ops * world / (e_ms * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": 5 * n_ops, "d2h_bytes_per_step": n_ops + 5 * n_vars + 8,
               "ms_per_step": e_ms, "api": "amc_check_trace_host",
               "chunk_ops": args.e2e_chunk or (1 << 25),
               "mode": "pinned host buffers; copies in, checks and copies out of chunks overlapped"}
        if amc.sync_status() != 0:
            raise RuntimeError("device error during e2e steps")
        # the host-buffer check must agree with the device-buffer one
        if not (torch.equal(hout["final_status"], out["final_status"].cpu()) and
                torch.equal(hout["var_first_fault"], out["var_first_fault"].cpu()) and
                torch.equal(hout["first_fault"], out["first_fault"].cpu()) and
                torch.equal(hout["step_status"][::997], out["step_status"][::997].cpu())):
            raise RuntimeError("host-buffer check differs from the device-buffer check")
        host_copy = (ks_h.numpy(), var_h.numpy())
    else:
        host_copy = None

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu:
        if host_copy is None:
            m = 1 << 26
            host_copy = (ks[:m].cpu().numpy(), var[:m].cpu().numpy())
        cpu = cpu_baseline(host_copy[0], host_copy[1], n_vars, args.cpu_seconds)
        cpu_all = cpu_baseline_all(host_copy[0], host_copy[1], n_vars, args.cpu_seconds / 2, host_threads(args))

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": ms_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
                "config": {"workload": "zipf_trace", "n_ops": n_ops, "n_vars": n_vars, "zipf_s": 1.05,
                           "kind_mix": "r.40 w.20 Push.15 Pull.15 Noop.10", "seed": args.seed,
                           "l2": "inputs 5 B/op exceed L2, no flush",
                           "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
                "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                             "frac": achieved / peak, "peak_kind": peak_kind,
                             "frac_of_8tbs": achieved / 8000.0, "traffic": traffic,
                             "kernel": trace_kernels(n_ops, n_vars)[0], "kernel_ms": k_ms,
                             "algorithmic_bytes": alg_bytes},
                "gpu_launches": trace_kernels(n_ops, n_vars)[1] * args.steps,
                "clocks": clk, "e2e": e2e, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all}
    if world > 1:
        if rank == 0:
            print(json.dumps(line), flush=True)
        import torch.distributed as dist
        dist.destroy_process_group()
        return
    if args.workload == "all":
        # the other workloads, after the trace's buffers are released
        del ks, var, out, ws
        if not args.no_e2e:
            del ks_h, var_h, hout, hws
        host_copy = None
        import gc
        gc.collect()
        torch.cuda.empty_cache()
        line["configs"] = sub_records(args, amc, dev)
    print(json.dumps(line), flush=True)


def sub_records(args, amc, dev):
    out = {}
    for name, fn in (("uniform_4096", lambda: measure_uniform(args, amc, dev)),
                     ("vectorpu", lambda: measure_vectorpu(args, amc, dev)),
                     ("vectorpu_lifetimes", lambda: measure_lifetimes(args, amc, dev)),
                     ("trace_sizes", lambda: measure_sizes(args, amc, dev)),
                     ("programs", lambda: measure_programs(args, amc, dev)),
                     ("programs_guarded", lambda: measure_guarded(args, amc, dev)),
                     ("well_declared", lambda: measure_well_declared(args, amc, dev)),
                     ("kloc", lambda: measure_kloc(args, amc, dev)),
                     ("serve", lambda: measure_serve(args, amc, dev))):
        import torch
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as e:            # one sub-record's failure does not hide the others
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = time.perf_counter() - t0
        torch.cuda.empty_cache()
    return out


def ctypes_ptr(ev):
    import ctypes
    return ctypes.c_void_p(ev.cuda_event)


def timed(fn, steps, stream):
    import torch
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def host_threads(args):
    return args.threads if args.threads > 0 else len(os.sched_getaffinity(0))


def roofline(alg_bytes, ms, note=None, bound="hbm"):
    peak, kind = peaks()
    ach = alg_bytes / (ms * 1e-3) / 1e9
    r = {"bound": bound, "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "peak_kind": kind,
         "frac_of_8tbs": ach / 8000.0, "traffic": None, "algorithmic_bytes": int(alg_bytes)}
    if note:
        r["note"] = note
    return r


def timed_calls(fn, budget_s, min_calls=1):
    """Calls fn() repeatedly for about budget_s seconds; returns (calls, seconds)."""
    t0 = time.perf_counter()
    fn()
    one = max(time.perf_counter() - t0, 1e-6)
    reps = max(min_calls, int(budget_s / one))
    t0 = time.perf_counter()
    for _ in range(reps):
        fn()
    return reps, time.perf_counter() - t0


def measure_uniform(args, amc, dev):
    """16 variables, 4,096 uniform ops (seed 0): latency of one check."""
    import numpy as np
    import torch

    import oracle
    import workloads
    ks_np, var_np, nv = workloads.trace_uniform(0)
    n = len(ks_np)
    ks, var = torch.from_numpy(ks_np).to(dev), torch.from_numpy(var_np).to(dev)
    stream = torch.cuda.Stream()
    out = dict(step_status=torch.empty(n, dtype=torch.uint8, device=dev),
               final_status=torch.empty(nv, dtype=torch.uint8, device=dev),
               var_first_fault=torch.empty(nv, dtype=torch.int32, device=dev),
               first_fault=torch.empty(1, dtype=torch.int64, device=dev))
    ws = torch.empty(amc.trace_workspace_bytes(n, nv) + 256, dtype=torch.uint8, device=dev)
    ws = ws[(-ws.data_ptr()) % 256:]
    step = lambda: amc.check_trace(ks, var, nv, out=out, workspace=ws, stream=stream)
    for _ in range(20):
        step()
    assert amc.sync_status(stream) == 0
    reps = 1000
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    clocks = ClockSampler(0)
    clocks.start()
    torch.cuda.synchronize()
    for a, b in ev:
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    lat = sorted(a.elapsed_time(b) * 1e3 for a, b in ev)          # us, each check alone on its stream
    back = timed(step, reps, stream) * 1e3                          # us per check, back to back
    clk = clocks.stop()
    assert amc.sync_status(stream) == 0
    exp = oracle.check_trace(ks_np, var_np, nv)
    assert np.array_equal(out["step_status"].cpu().numpy(), exp[0]) and int(out["first_fault"].cpu()[0]) == exp[3]
    # end to end: pinned host buffers, copies inside the call
    ks_h, var_h = torch.from_numpy(ks_np).pin_memory(), torch.from_numpy(var_np).pin_memory()
    hws = torch.empty(amc.trace_host_workspace_bytes(n, nv, 0) + 256, dtype=torch.uint8, device=dev)
    hws = hws[(-hws.data_ptr()) % 256:]
    e2e_step = lambda: (amc.check_trace_host(ks_h, var_h, nv, workspace=hws, stream=stream), stream.synchronize())
    for _ in range(10):
        e2e_step()
    e_reps, e_s = timed_calls(e2e_step, 0.5, 100)
    r_cpu, t_cpu = timed_calls(lambda: oracle.check_trace(ks_np, var_np, nv), 1.0, 100)
    med = statistics.median(lat)
    alg = 6 * n + 5 * nv
    return {"workload": "uniform_trace", "n_ops": n, "n_vars": nv, "seed": 0,
            "us_per_check_median": med, "us_per_check_best": lat[0], "us_per_check_p99": lat[int(0.99 * len(lat))],
            "us_per_check_back_to_back": back, "checks": reps, "ops_per_s": n / (med * 1e-6),
            "roofline": roofline(alg, med * 1e-3, bound="latency",
                                 note="24,656 algorithmic bytes per check: latency-bound, the fraction is not "
                                      "meaningful"),
            "gpu_launches_per_check": trace_kernels(n, nv)[1],
            "e2e": {"us_per_check": e_s / e_reps * 1e6, "api": "amc_check_trace_host",
                    "h2d_bytes_per_step": 5 * n, "d2h_bytes_per_step": n + 5 * nv + 8,
                    "mode": "pinned host buffers, call + stream synchronise per check"},
            "cpu_baseline": {"value": r_cpu * n / t_cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "us_per_check": t_cpu / r_cpu * 1e6,
                             "sample": f"the whole trace, {r_cpu} passes, single thread"},
            "clocks": clk}


def measure_vectorpu(args, amc, dev):
    """2^24 VectorPU calls (seed 2): translation + guarded check per step."""
    import numpy as np
    import torch

    import oracle
    import workloads
    w = workloads.vectorpu_calls(seed=2)
    d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in w.items()}
    A = d["arr_start"].numel()
    n_calls = d["call_side"].numel()
    n_opnd = d["opnd_array"].numel()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        tr = amc.translate_vectorpu(d["arr_start"], d["arr_len"], d["call_side"], d["call_off"], d["opnd_array"],
                                    d["opnd_mode"], stream=stream)
        n = tr["n"]
        tout = dict(kind_side=tr["kind_side"], var=tr["var"], call_first_op=tr["call_first_op"], n_dev=tr["n_dev"])
        out = dict(step_status=torch.empty(n, dtype=torch.uint8, device=dev),
                   final_status=torch.empty(2 * A, dtype=torch.uint8, device=dev),
                   var_first_fault=torch.empty(2 * A, dtype=torch.int32, device=dev),
                   first_fault=torch.empty(1, dtype=torch.int64, device=dev))
        ws = torch.empty(amc.trace_workspace_bytes(n, 2 * A, guarded=True) + 256, dtype=torch.uint8, device=dev)
        ws = ws[(-ws.data_ptr()) % 256:]

        def step():
            r = amc.translate_vectorpu(d["arr_start"], d["arr_len"], d["call_side"], d["call_off"],
                                       d["opnd_array"], d["opnd_mode"], known_n=n, out=tout, stream=stream)
            amc.check_trace(r["kind_side"], r["var"], 2 * A, guarded=True, out=out, workspace=ws, stream=stream)

        for _ in range(max(3, args.warmup)):
            step()
        assert amc.sync_status(stream) == 0
        clocks = ClockSampler(0)
        clocks.start()
        ms = timed(step, args.sub_steps, stream)
        clk = clocks.stop()
        assert amc.sync_status(stream) == 0
        assert int(tout["n_dev"].item()) == n
    # oracle: the first calls, about sub_cpu_seconds of one core
    k = 1 << 14
    while True:
        sub = dict(w)
        sub["call_side"] = w["call_side"][:k]
        sub["call_off"] = w["call_off"][:k + 1]
        m = int(w["call_off"][k])
        sub["opnd_array"] = w["opnd_array"][:m]
        sub["opnd_mode"] = w["opnd_mode"][:m]
        t0 = time.perf_counter()
        res = oracle.vectorpu(**sub)
        dt = time.perf_counter() - t0
        if dt > args.sub_cpu_seconds / 4 or k >= n_calls:
            break
        k = min(n_calls, k * 4)
    # the oracle's statuses of those calls are the GPU's first statuses
    ns = len(res["step_status"])
    assert np.array_equal(out["step_status"][:ns].cpu().numpy(), res["step_status"])
    alg = 8 * A + n_calls + 4 * (n_calls + 1) + 5 * n_opnd + n + 5 * 2 * A
    return {"workload": "vectorpu_calls", "n_arrays": A, "n_calls": n_calls, "operands": n_opnd, "statements": n,
            "seed": 2, "ms_per_step": ms, "statements_per_s": n / (ms * 1e-3), "calls_per_s": n_calls / (ms * 1e-3),
            "roofline": roofline(alg, ms, note="algorithmic bytes: arrays, calls and operands in, one status per "
                                               "translated statement and 5 B per variable out"),
            "gpu_launches_per_step": vectorpu_launches(n, 2 * A),
            "cpu_baseline": {"value": ns / dt, "unit": "statements/s", "calls_per_s": k / dt, "cores": 1,
                             "kind": "oracle",
                             "sample": f"the first {k} calls ({ns} statements), single thread ({dt:.1f} s)"},
            "clocks": clk}


def measure_lifetimes(args, amc, dev):
    """2^24 VectorPU calls over 16 vectors and 65,536 pvectors created and
    deleted during the run (seed 6): translation with live overlap sets and
    creation records, then the check with inherited statuses (two guarded
    passes) per step."""
    import numpy as np
    import torch

    import oracle
    import workloads
    w = workloads.vectorpu_lifetimes(seed=6)
    d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in w.items()}
    A = d["arr_start"].numel()
    n_calls = d["call_side"].numel()
    n_opnd = d["opnd_array"].numel()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        args_tr = (d["arr_start"], d["arr_len"], d["arr_parent"], d["arr_born"], d["arr_died"], d["call_side"],
                   d["call_off"], d["opnd_array"], d["opnd_mode"])
        tr = amc.translate_vectorpu_lifetimes(*args_tr, stream=stream)
        n, pairs = tr["n"], tr["max_pairs"]
        tout = dict(kind_side=tr["kind_side"], var=tr["var"], call_first_op=tr["call_first_op"],
                    arr_probe=tr["arr_probe"], n_dev=tr["n_dev"])
        out = dict(step_status=torch.empty(n, dtype=torch.uint8, device=dev),
                   final_status=torch.empty(2 * A, dtype=torch.uint8, device=dev),
                   var_first_fault=torch.empty(2 * A, dtype=torch.int32, device=dev),
                   first_fault=torch.empty(1, dtype=torch.int64, device=dev))
        L = amc.lib()
        ws = torch.empty(L.amc_check_inherited_trace_workspace(n, A) + 256, dtype=torch.uint8, device=dev)
        ws = ws[(-ws.data_ptr()) % 256:]

        def step():
            r = amc.translate_vectorpu_lifetimes(*args_tr, max_pairs=pairs, known_n=n, out=tout, stream=stream)
            amc.check_inherited_trace(r["kind_side"], r["var"], A, d["arr_parent"], r["arr_probe"], out=out,
                                      workspace=ws, stream=stream)

        for _ in range(max(3, args.warmup)):
            step()
        assert amc.sync_status(stream) == 0
        clocks = ClockSampler(0)
        clocks.start()
        ms = timed(step, args.sub_steps, stream)
        clk = clocks.stop()
        assert amc.sync_status(stream) == 0
        assert int(tout["n_dev"].item()) == n
    # oracle: the first k calls (lifetimes clipped to them), about
    # sub_cpu_seconds of one core; its statuses before call k - 1 are the GPU's
    k = 1 << 12
    while True:
        sub = dict(w)
        sub["arr_born"] = np.minimum(w["arr_born"], k - 1).astype(np.int32)
        sub["arr_died"] = np.maximum(np.minimum(w["arr_died"], k), sub["arr_born"] + 1).astype(np.int32)
        sub["call_side"] = w["call_side"][:k]
        sub["call_off"] = w["call_off"][:k + 1]
        m = int(w["call_off"][k])
        sub["opnd_array"] = w["opnd_array"][:m]
        sub["opnd_mode"] = w["opnd_mode"][:m]
        t0 = time.perf_counter()
        res = oracle.vectorpu_lifetimes(**sub)
        dt = time.perf_counter() - t0
        if dt > args.sub_cpu_seconds / 4 or k >= n_calls:
            break
        k = min(n_calls, k * 4)
    ns = int(res["call_first_op"][k - 1])
    assert np.array_equal(out["step_status"][:ns].cpu().numpy(), res["step_status"][:ns])
    alg = 20 * A + n_calls + 4 * (n_calls + 1) + 5 * n_opnd + n + 8 * A + 5 * 2 * A
    return {"workload": "vectorpu_lifetimes", "n_vectors": 16, "n_pvectors": A - 16, "n_calls": n_calls,
            "operands": n_opnd, "statements": n, "overlap_list_entries": pairs, "seed": 6, "ms_per_step": ms,
            "statements_per_s": n / (ms * 1e-3), "calls_per_s": n_calls / (ms * 1e-3),
            "roofline": roofline(alg, ms, note="algorithmic bytes: arrays (range, vector, lifetime), calls and "
                                               "operands in; one status per translated statement, the creation "
                                               "records and 5 B per variable out"),
            "gpu_launches_per_step": lifetimes_launches(A, n_calls, n),
            "cpu_baseline": {"value": ns / dt, "unit": "statements/s", "calls_per_s": k / dt, "cores": 1,
                             "kind": "oracle",
                             "sample": f"the first {k} calls (lifetimes clipped to them; {ns} statements compared), "
                                       f"single thread ({dt:.1f} s)"},
            "clocks": clk}


def measure_sizes(args, amc, dev):
    """The trace check away from the headline size: Zipf(1.05) traces over
    2^20 variables (the headline kind mix) of 2^24, 2^26 and 2^28 ops, and a
    2^30-op low-fault trace (r .02 w .60 Push .05 Pull .05 Noop .28), each
    timed over sub_steps checks after the first call of its size class has
    timed the candidate paths."""
    import torch

    import workloads
    nv = 1 << 20
    cases = [("zipf_2p24", 1 << 24, workloads.KIND_MIX), ("zipf_2p26", 1 << 26, workloads.KIND_MIX),
             ("zipf_2p28", 1 << 28, workloads.KIND_MIX), ("low_fault_2p30", 1 << 30, (0.02, 0.60, 0.05, 0.05, 0.28))]
    out = {}
    stream = torch.cuda.Stream()
    for name, n, mix in cases:
        with torch.cuda.stream(stream):
            ks, var = workloads.trace_zipf(n, nv, seed=1, device=dev, kind_mix=mix)
            res = dict(step_status=torch.empty(n, dtype=torch.uint8, device=dev),
                       final_status=torch.empty(nv, dtype=torch.uint8, device=dev),
                       var_first_fault=torch.empty(nv, dtype=torch.int32, device=dev),
                       first_fault=torch.empty(1, dtype=torch.int64, device=dev))
            ws = torch.empty(amc.trace_workspace_bytes(n, nv) + 256, dtype=torch.uint8, device=dev)
            ws = ws[(-ws.data_ptr()) % 256:]
            step = lambda: amc.check_trace(ks, var, nv, out=res, workspace=ws, stream=stream)
            for _ in range(max(3, args.warmup)):
                step()
            assert amc.sync_status(stream) == 0
            clocks = ClockSampler(0)
            clocks.start()
            ms = timed(step, args.sub_steps, stream)
            clk = clocks.stop()
            assert amc.sync_status(stream) == 0
            stuck = int((res["step_status"] == 4).sum().item())
            path, launches = amc.trace_plan(n, nv)
            alg = 6 * n + 5 * nv
            out[name] = {"n_ops": n, "n_vars": nv, "kind_mix": list(mix), "seed": 1, "ms_per_check": ms,
                         "ops_per_s": n / (ms * 1e-3), "stuck_fraction": stuck / n, "path": path,
                         "gpu_launches_per_check": launches,
                         "roofline": roofline(alg, ms, note="6 B per op, 5 B per variable; the span of the "
                                                            "whole check (every kernel)"),
                         "l2": "inputs exceed L2" if 5 * n > (129 << 20) else "inputs fit in L2 (warm)",
                         "clocks": clk}
            del ks, var, res, ws
            torch.cuda.empty_cache()
    return out


def measure_programs(args, amc, dev):
    """100,000 programs (seed 3): the batched persistent launch (graph replay)
    against one launch per program through the same entry point."""
    import ctypes
    import threading

    import numpy as np
    import torch

    import oracle
    import workloads
    b = workloads.programs(n_progs=args.n_progs)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    tok, pay, off, nv = t(b["tok"]), t(b["payload"]), t(b["prog_tok_off"]), t(b["prog_nvars"])
    vo = torch.zeros(nv.numel() + 1, dtype=torch.int64, device=dev)
    torch.cumsum(nv.to(torch.int64), 0, out=vo[1:])
    n_tok = tok.numel()
    P = nv.numel()
    total_vars = int(vo[-1])
    leaf = int(b["n_leaf"].sum())
    out = dict(step_mask=torch.empty(n_tok, dtype=torch.uint8, device=dev),
               final_mask=torch.empty(total_vars, dtype=torch.uint8, device=dev),
               prog_first_fault=torch.empty(P, dtype=torch.int64, device=dev))
    stream = torch.cuda.Stream()
    L = amc.lib()
    ws = torch.empty(L.amc_check_batch_workspace(n_tok, P, total_vars) + 256, dtype=torch.uint8, device=dev)
    ws = ws[(-ws.data_ptr()) % 256:]
    with torch.cuda.stream(stream):
        batched = lambda: amc.check_batch(tok, pay, off, nv, vo, graph_capture=True, out=out, workspace=ws,
                                          stream=stream)
        for _ in range(max(3, args.warmup)):
            batched()
        assert amc.sync_status(stream) == 0
        clocks = ClockSampler(0)
        clocks.start()
        ms_b = timed(batched, args.sub_steps, stream)
        clk = clocks.stop()
        assert amc.sync_status(stream) == 0
        step_b = out["step_mask"].cpu().numpy()
        plain = None
        k = min(args.plain_progs, P)
        if k > 0:
            # one launch per program (no graph) over the first k programs, each
            # program rebased to its own tokens (offsets [0, len]) with its own
            # small workspace, launched round-robin on PLAIN_STREAMS streams so
            # that up to that many programs run at once
            sp = [torch.cuda.Stream() for _ in range(PLAIN_STREAMS)]
            V = lambda x: ctypes.c_void_p(x)
            offs = b["prog_tok_off"]
            lens = np.diff(offs[:k + 1]).astype(np.int64)
            rel = np.zeros((k, 2), np.int64)
            rel[:, 1] = lens
            rel_d = t(rel.reshape(-1))
            wsz = int(L.amc_check_batch_workspace(int(lens.max()), 1, int(b["prog_nvars"][:k].max())))
            wss = []
            for _ in range(PLAIN_STREAMS):
                w1 = torch.empty(wsz + 256, dtype=torch.uint8, device=dev)
                wss.append(w1[(-w1.data_ptr()) % 256:])
            sm_p, fm_p, pf_p = out["step_mask"].data_ptr(), out["final_mask"].data_ptr(), \
                out["prog_first_fault"].data_ptr()

            def plain_run():
                for x in sp:
                    x.wait_stream(stream)
                for i in range(k):
                    j = i % PLAIN_STREAMS
                    a0 = int(offs[i])
                    rc = L.amc_check_batch(V(tok.data_ptr() + a0), V(pay.data_ptr() + 4 * a0), V(rel_d.data_ptr() + 16 * i),
                                           V(nv.data_ptr() + 4 * i), V(vo.data_ptr() + 8 * i), 1, int(lens[i]),
                                           V(sm_p + a0), V(fm_p), V(pf_p + 8 * i), 0, V(wss[j].data_ptr()), wsz,
                                           V(sp[j].cuda_stream))
                    assert rc == 0, rc
                for x in sp:
                    stream.wait_stream(x)

            plain_run()
            assert amc.sync_status(stream) == 0
            ms_p = timed(plain_run, 1, stream)
            assert amc.sync_status(stream) == 0
            tk = int(offs[k])
            assert np.array_equal(out["step_mask"][:tk].cpu().numpy(), step_b[:tk])
            plain = {"programs": k, "tokens": tk, "ms": ms_p, "value": tk / (ms_p * 1e-3),
                     "ms_per_program": ms_p / k, "streams": PLAIN_STREAMS,
                     "mode": f"one amc_check_batch launch per program (no graph), the first {k} programs of the "
                             f"batch, each rebased to its own tokens with its own workspace, round-robin on "
                             f"{PLAIN_STREAMS} streams"}
    # oracle: programs sharded over the host threads, and one thread
    T = host_threads(args)
    to_np = b["prog_tok_off"]

    def oracle_range(lo, hi):
        a0, a1 = int(to_np[lo]), int(to_np[hi])
        return oracle.check_batch(b["tok"][a0:a1], b["payload"][a0:a1], to_np[lo:hi + 1] - a0, b["prog_nvars"][lo:hi])

    k1 = 256
    while True:
        t0 = time.perf_counter()
        r1 = oracle_range(0, k1)
        dt1 = time.perf_counter() - t0
        if dt1 > args.sub_cpu_seconds / 4 or k1 >= P:
            break
        k1 = min(P, k1 * 4)
    assert np.array_equal(r1[0], step_b[:int(to_np[k1])])
    kT = min(P, k1 * T)
    bounds = np.linspace(0, kT, T + 1).astype(int)
    th = [threading.Thread(target=oracle_range, args=(int(bounds[i]), int(bounds[i + 1]))) for i in range(T)]
    t0 = time.perf_counter()
    for x in th:
        x.start()
    for x in th:
        x.join()
    dtT = time.perf_counter() - t0
    tok1, tokT = int(to_np[k1]), int(to_np[kT])
    alg = 5 * n_tok + n_tok + 8 * (P + 1) * 2 + 4 * P + total_vars + 8 * P
    return {"workload": "programs", "n_progs": P, "tokens": n_tok, "leaf_ops": leaf, "seed": 3,
            "ms_per_step": ms_b, "tokens_per_s": n_tok / (ms_b * 1e-3), "leaf_ops_per_s": leaf / (ms_b * 1e-3),
            "mode": "batched persistent launch, CUDA graph replay",
            "plain": plain, "batched_over_plain": None if plain is None else (n_tok / ms_b) / (plain["tokens"] / plain["ms"]),
            "roofline": roofline(alg, ms_b, note="algorithmic bytes: 5 B per token in, 1 B per token out, CSR "
                                                  "offsets, one mask per variable"),
            "gpu_launches_per_step": batch_launches(n_tok),
            "cpu_baseline": {"value": tok1 / dt1, "unit": "tokens/s", "cores": 1, "kind": "oracle",
                             "sample": f"the first {k1} programs ({tok1} tokens), single thread ({dt1:.1f} s)"},
            "cpu_baseline_all_cores": {"value": tokT / dtT, "unit": "tokens/s", "cores": T, "kind": "oracle",
                                       "sample": f"the first {kT} programs ({tokT} tokens) sharded by program over "
                                                 f"{T} threads ({dtT:.1f} s)"},
            "clocks": clk}


def batch_launches(n_tokens):
    """Kernels of one batched relation-mode check (longest-first queue):
    bucket count, scan and order; when the batch is longer than the split
    length (so that some program may be split) also the slot offsets, the
    cuts, the relation reset, the ordered unit offsets, the reduce phase and
    the carry; then the apply phase."""
    split = int(os.environ.get("AMC_BATCH_SPLIT", "65536"))
    return 3 + 1 if n_tokens <= split else 3 + 3 + 1 + 1 + 1 + 1


def measure_guarded(args, amc, dev):
    """20,000 programs over 16-256 variables whose If conditions test a guard
    variable (seed 7): the path-sensitive relation mode, one launch sequence
    per step."""
    import numpy as np
    import torch

    import oracle
    import workloads
    b = workloads.programs_guarded()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    tok, pay, off, nv, gd = t(b["tok"]), t(b["payload"]), t(b["prog_tok_off"]), t(b["prog_nvars"]), t(b["prog_guard"])
    vo = torch.zeros(nv.numel() + 1, dtype=torch.int64, device=dev)
    torch.cumsum(nv.to(torch.int64), 0, out=vo[1:])
    n_tok, P, total_vars = tok.numel(), nv.numel(), int(vo[-1])
    out = dict(step_mask=torch.empty(n_tok, dtype=torch.uint8, device=dev),
               final_mask=torch.empty(total_vars, dtype=torch.uint8, device=dev),
               prog_first_fault=torch.empty(P, dtype=torch.int64, device=dev))
    L = amc.lib()
    ws = torch.empty(L.amc_check_batch_guarded_workspace(n_tok, P, total_vars) + 256, dtype=torch.uint8, device=dev)
    ws = ws[(-ws.data_ptr()) % 256:]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        step = lambda: amc.check_batch_guarded(tok, pay, off, nv, gd, vo, out=out, workspace=ws, stream=stream)
        for _ in range(max(3, args.warmup)):
            step()
        assert amc.sync_status(stream) == 0
        clocks = ClockSampler(0)
        clocks.start()
        ms = timed(step, args.sub_steps, stream)
        clk = clocks.stop()
        assert amc.sync_status(stream) == 0
        got = out["step_mask"].cpu().numpy()
    to_np = b["prog_tok_off"]
    k1 = 256
    while True:
        a1 = int(to_np[k1])
        t0 = time.perf_counter()
        r1 = oracle.check_batch_guarded(b["tok"][:a1], b["payload"][:a1], to_np[:k1 + 1], b["prog_nvars"][:k1],
                                        b["prog_guard"][:k1])
        dt1 = time.perf_counter() - t0
        if dt1 > args.sub_cpu_seconds / 4 or k1 >= P:
            break
        k1 = min(P, k1 * 4)
    assert np.array_equal(r1[0], got[:a1])
    ops = (b["tok"] & 15) <= 5
    alg = 5 * n_tok + n_tok + 8 * (P + 1) * 2 + 8 * P + total_vars + 8 * P
    return {"workload": "programs_guarded", "n_progs": P, "tokens": n_tok, "seed": 7, "ms_per_step": ms,
            "tokens_per_s": n_tok / (ms * 1e-3),
            "unreachable_op_fraction": float(((got == 0) & ops).sum() / max(1, ops.sum())),
            "roofline": roofline(alg, ms, note="algorithmic bytes: 5 B per token in, 1 B per token out, CSR "
                                               "offsets and guards, one mask per variable"),
            "gpu_launches_per_step": 4,
            "cpu_baseline": {"value": a1 / dt1, "unit": "tokens/s", "cores": 1, "kind": "oracle",
                             "sample": f"the first {k1} programs ({a1} tokens), single thread ({dt1:.1f} s)"},
            "clocks": clk}


def measure_well_declared(args, amc, dev):
    """2^20 calls AM{S} (seed 5): the static well-declaredness check."""
    import numpy as np
    import torch

    import oracle
    import workloads
    w = workloads.wd_calls()
    d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in w.items()}
    C = d["call_tok_off"].numel() - 1
    T = d["tok"].numel()
    D = d["am_array"].numel()
    stream = torch.cuda.Stream()
    out = dict(violations=torch.empty(C, dtype=torch.int32, device=dev),
               first_bad=torch.empty(C, dtype=torch.int64, device=dev),
               first_unmet=torch.empty(C, dtype=torch.int32, device=dev))
    step = lambda: amc.check_well_declared(d["arr_loc_off"], d["loc_owner"], d["call_tok_off"], d["tok"],
                                           d["payload"], d["call_am_off"], d["am_array"], d["am_mode"], out=out,
                                           stream=stream)
    for _ in range(max(3, args.warmup)):
        step()
    assert amc.sync_status(stream) == 0
    clocks = ClockSampler(0)
    clocks.start()
    ms = timed(step, args.sub_steps, stream)
    clk = clocks.stop()
    assert amc.sync_status(stream) == 0
    reps, dt = timed_calls(lambda: oracle.well_declared(**w), args.sub_cpu_seconds, 1)
    exp = oracle.well_declared(**w)
    assert np.array_equal(out["violations"].cpu().numpy().astype(np.uint32), exp[0])
    assert np.array_equal(out["first_bad"].cpu().numpy(), exp[1])
    assert np.array_equal(out["first_unmet"].cpu().numpy(), exp[2])
    alg = 5 * T + 5 * D + 16 * (C + 1) + 16 * C + 8 * w["arr_loc_off"].size + 4 * w["loc_owner"].size
    return {"workload": "wd_calls", "n_calls": C, "tokens": T, "declarations": D, "seed": 5,
            "ms_per_step": ms, "calls_per_s": C / (ms * 1e-3), "tokens_per_s": T / (ms * 1e-3),
            "violating_calls": int((exp[0] != 0).sum()),
            "roofline": roofline(alg, ms, note="algorithmic bytes: tokens, declarations and call offsets in, "
                                               "three words per call out"),
            "gpu_launches_per_step": 1,
            "cpu_baseline": {"value": reps * C / dt, "unit": "calls/s", "cores": 1, "kind": "oracle",
                             "sample": f"the whole workload, {reps} pass(es), single thread ({dt:.1f} s)"},
            "clocks": clk}


def measure_kloc(args, amc, dev):
    """Traces over k = 4 memory locations: 2^28 ops over 2^20 variables, Zipf
    ids as the headline trace, kinds r .40 / w .20 / copy .30 / Noop .10 with
    the locations drawn uniformly (seed 6)."""
    import numpy as np
    import torch

    import oracle
    import workloads
    k, n, nv = 4, 1 << 28, 1 << 20
    g = torch.Generator(device=dev)
    g.manual_seed(6)
    ks, var = workloads.trace_zipf(n, nv, seed=6, device=dev)      # ids; the op bytes are redrawn below
    del ks
    u = torch.rand(n, device=dev, generator=g)
    kind = torch.bucketize(u, torch.tensor([0.4, 0.6, 0.9], device=dev))
    a = torch.randint(0, k, (n,), device=dev, generator=g)
    b = (a + torch.randint(1, k, (n,), device=dev, generator=g)) % k
    op = torch.where(kind == 3, torch.full_like(a, 3),
                     torch.where(kind == 2, kind | a << 2 | b << 5, kind | a << 2)).to(torch.uint8)
    del u, kind, a, b
    stream = torch.cuda.Stream()
    out = dict(step_status=torch.empty(n, dtype=torch.uint8, device=dev),
               final_status=torch.empty(nv, dtype=torch.uint8, device=dev),
               var_first_fault=torch.empty(nv, dtype=torch.int32, device=dev),
               first_fault=torch.empty(1, dtype=torch.int64, device=dev))
    ws = torch.empty(amc.lib().amc_check_trace_k_workspace(n, nv) + 256, dtype=torch.uint8, device=dev)
    ws = ws[(-ws.data_ptr()) % 256:]
    step = lambda: amc.check_trace_k(op, var, nv, k, out=out, workspace=ws, stream=stream)
    for _ in range(max(3, args.warmup)):
        step()
    assert amc.sync_status(stream) == 0
    clocks = ClockSampler(0)
    clocks.start()
    ms = timed(step, args.sub_steps, stream)
    clk = clocks.stop()
    assert amc.sync_status(stream) == 0
    m = 1 << 24
    op_h, var_h = op[:m].cpu().numpy(), var[:m].cpu().numpy()
    reps, dt = timed_calls(lambda: oracle.check_trace_k(op_h, var_h, nv, k), args.sub_cpu_seconds, 1)
    exp = oracle.check_trace_k(op_h, var_h, nv, k)
    assert np.array_equal(out["step_status"][:m].cpu().numpy(), exp[0])
    alg = 6 * n + 5 * nv
    return {"workload": "kloc_trace", "k": k, "n_ops": n, "n_vars": nv, "seed": 6, "ms_per_step": ms,
            "ops_per_s": n / (ms * 1e-3),
            "roofline": roofline(alg, ms, note="algorithmic bytes: 5 B per op in, 1 B per op out, 5 B per variable"),
            "gpu_launches_per_step": 11,
            "cpu_baseline": {"value": reps * m / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"the first {m} ops, {reps} pass(es), single thread ({dt:.1f} s)"},
            "clocks": clk}


def phase_summary(phases):
    """Median / p99 of the server's queue wait (submit to admission) and service
    time (admission to done) in ms, for results as status codes (traces on
    sessions of single statuses) and as masks (programs, and traces after a
    program with constructs)."""
    import numpy as np
    out = {}
    for kind, name in ((0, "code_results"), (1, "mask_results")):
        q = np.array([p[0] for p in phases if p[2] == kind]) * 1e3
        sv = np.array([p[1] for p in phases if p[2] == kind]) * 1e3
        n = np.array([p[3] for p in phases if p[2] == kind])
        if q.size:
            out[name] = {"queue_p50": float(np.percentile(q, 50)), "queue_p99": float(np.percentile(q, 99)),
                         "service_p50": float(np.percentile(sv, 50)), "service_p99": float(np.percentile(sv, 99)),
                         "service_sum_s": float(sv.sum() / 1e3), "items": int(n.sum()), "requests": int(q.size)}
    return out


def measure_serve(args, amc, dev):
    """Open-loop Poisson arrivals into the continuous-batching server.  Every
    request is prepared before the clock starts: traces are slices of pinned op
    pools, one per session size (var ids uniform over the session's variables),
    submitted with AMC_REQ_BORROW; programs are generated in advance.  Latency
    = poll-visible completion - scheduled arrival; submission stops after
    --serve-seconds per rate and the requests not submitted by then are
    counted."""
    import threading

    import numpy as np
    import torch

    # the submitter and the poller share the interpreter: switch often
    sys.setswitchinterval(1e-4)

    import workloads
    P = 1 << 24
    grid = workloads.SERVE_NV_GRID
    g = torch.Generator(device=dev)
    g.manual_seed(4)
    kcdf = torch.tensor(np.cumsum(workloads.KIND_MIX)[:-1], dtype=torch.float32, device=dev)
    pools = {}
    for nv in grid:
        kind = torch.bucketize(torch.rand(P, device=dev, generator=g), kcdf, right=True)
        side = torch.randint(0, 2, (P,), device=dev, generator=g)
        ks = (kind | side << 4).to(torch.uint8).cpu().pin_memory()
        var = torch.randint(0, nv, (P,), device=dev, generator=g, dtype=torch.int32).cpu().pin_memory()
        pools[nv] = (ks, var)
    results = {}
    clocks = ClockSampler(0)
    clocks.start()
    for rate in [float(x) for x in args.rates.split(",")]:
        sch = workloads.serve_schedule(rate, n_requests=args.serve_requests, seed=4)
        reqs = []
        for i in range(len(sch["arrival"])):
            nv = int(sch["nv"][i])
            if sch["kind"][i] == 0:
                a, n = int(sch["offset"][i]), int(sch["n_ops"][i])
                ks, var = pools[nv]
                reqs.append((int(sch["session"][i]), 0, nv, ks[a:a + n], var[a:a + n], True, float(sch["arrival"][i])))
            else:
                b = workloads.programs(1, seed=44, first=int(sch["prog_index"][i]), vars_lo=nv, vars_hi=nv)
                reqs.append((int(sch["session"][i]), 1, nv, b["tok"], b["payload"], False, float(sch["arrival"][i])))
        with amc.Server(mem_budget_bytes=32 << 30, max_slots=32) as srv:
            tickets = {}
            lat, errs = [], [0]
            items = [0]
            lock = threading.Lock()
            done_flag = [False]
            backp = [0]

            phases = []

            def poller():
                # the server reports what finished; only those are read (a
                # ticket can finish before the submitter has recorded it)
                early = {}
                while True:
                    with lock:
                        if done_flag[0] and not tickets:
                            return
                    for tk in srv.completed():
                        r = srv.poll(tk)
                        early[tk] = (time.perf_counter(), len(r["status"]), r["error"] != 0)
                        phases.append((r["t_admit"] - r["t_submit"], r["t_done"] - r["t_admit"],
                                       1 if r["is_mask"] else 0, len(r["status"])))
                    with lock:
                        for tk in [t for t in early if t in tickets]:
                            now, n_items, bad = early.pop(tk)
                            lat.append(now - (t0 + tickets.pop(tk)))
                            items[0] += n_items
                            errs[0] += bad
                    if time.perf_counter() > drain_deadline[0]:
                        return
                    time.sleep(2e-5)

            drain_deadline = [float("inf")]
            th = threading.Thread(target=poller)
            t0 = time.perf_counter() + 0.05
            th.start()
            submitted = 0
            last_submit = t0
            for sid, kind, nv, a, bb, borrow, at in reqs:
                # wait for the scheduled arrival without holding the interpreter
                while (wait := t0 + at - time.perf_counter()) > 0:
                    time.sleep(wait if wait > 2e-4 else 0)
                if time.perf_counter() - t0 > args.serve_seconds:
                    break
                while (tk := srv.submit(sid, kind, nv, a, bb, borrow=borrow)) is None:
                    backp[0] += 1
                    time.sleep(1e-5)
                last_submit = time.perf_counter()
                submitted += 1
                with lock:
                    tickets[tk] = at
            drain_deadline[0] = time.perf_counter() + args.serve_drain_seconds
            done_flag[0] = True
            th.join()
            wall = time.perf_counter() - t0
            unfinished = len(tickets)
        lat_ms = np.array(lat) * 1e3
        span = reqs[submitted - 1][6] if submitted else 0.0
        results[str(int(rate))] = {"p50_ms": float(np.percentile(lat_ms, 50)) if len(lat) else None,
                                   "p99_ms": float(np.percentile(lat_ms, 99)) if len(lat) else None,
                                   "max_ms": float(lat_ms.max()) if len(lat) else None,
                                   "requests": len(reqs), "submitted": submitted, "completed": len(lat),
                                   "unfinished_at_deadline": unfinished, "errors": errs[0],
                                   "offered_rate": submitted / span if span > 0 else None,
                                   "achieved_submit_rate": submitted / max(last_submit - t0, 1e-9),
                                   "backpressured_submits": backp[0],
                                   "program_requests": sum(1 for x in reqs[:submitted] if x[1] == 1),
                                   "items_per_s": items[0] / wall, "wall_s": wall,
                                   "server_phases_ms": phase_summary(phases)}
    clk = clocks.stop()
    del pools
    return {"workload": "serve", "rates_req_per_s": args.rates, "requests_per_rate": args.serve_requests,
            "slots": 32, "budget_gb": 32, "seed": 4,
            "sessions": "1-64 requests over n_vars drawn from 32 evenly spaced values in 64..4,032; kind drawn per "
                        "request (half programs, half traces of 2^10-2^24 ops)",
            "traces": "slices of pinned op pools (one per session size), submitted without a copy (AMC_REQ_BORROW)",
            "latency": "poll-visible completion minus scheduled arrival (open loop)",
            "by_rate": results, "clocks": clk}


def radix_passes(key_range):
    """Passes of the library's 7-bit LSD radix sort for keys below key_range."""
    kb = 1
    while kb < 31 and (1 << kb) < key_range:
        kb += 1
    return (kb + 6) // 7


def overlap_launches(n_arrays):
    """Kernels that build the overlap lists: keys, the sort by range start
    (three kernels per radix pass), the counting sweep, a three-kernel scan,
    the total, the cursor reset, the filling sweep, two sorts of the pairs,
    the copy and the overflow clear."""
    return 1 + 3 * radix_passes(2 ** 31 - 1) + 1 + 3 + 1 + 1 + 1 + 2 * 3 * radix_passes(n_arrays) + 1 + 1


def guarded_check_launches(n_statements, n_vars):
    """Kernels of one guarded check (two scan passes): the reduce / carry /
    apply path where the size rule takes it for a trace of that length (5
    kernels up to 8,192 variables -- warp batches and a two-level carry --
    else 3) in each pass, or the scan kernel plus, in the second pass, the
    final-status kernel."""
    import paper_1910_11110_gb300 as amc
    path, n = amc.trace_plan(n_statements, n_vars)
    if path in ("warp_dense", "dense"):
        return 2 * n
    return 1 + 2


def vectorpu_launches(n_statements, n_vars):
    """Kernels of one translation + guarded check: the overlap lists, counts,
    a three-kernel scan, emission and the total, then the guarded check."""
    return overlap_launches(n_vars // 2) + 1 + 3 + 1 + 1 + guarded_check_launches(n_statements, n_vars)


def lifetimes_launches(n_arrays, n_calls, n_statements):
    """Kernels of one lifetimes translation + inherited check: the overlap
    lists, the lifetimes check and the sort by creation call, counts, scan,
    emission and the total; then two guarded checks with the inheritance
    kernel between them."""
    births = 1 + 3 * radix_passes(n_calls + 1)
    return (overlap_launches(n_arrays) + births + 1 + 3 + 1 + 1 +
            2 * guarded_check_launches(n_statements, 2 * n_arrays) + 1)


TRACE_PATH_TEXT = {
    "small": "small_trace_kernel (one CTA: fold per warp stretch, carry per variable, apply)",
    "warp_dense": "warp reduce + carry + apply kernels",
    "dense": "dense reduce + carry + apply kernels",
    "prefix": "prefix (dense reduce + carry + apply) + scan_trace_kernel",
    "epochs": ("first part: sorted check (radix sort by variable + segmented scan); epochs to 4x their start: "
               "tail_filter_kernel + gather + bucket check of the candidates (one radix pass, a CTA per bucket)"),
    "scan": "scan_trace_kernel",
}


def trace_kernels(n_ops, n_vars, has_init=False):
    """(what the timed span covers, kernels launched per check) for the next
    amc_check_trace of these sizes, as the library reports it
    (amc_check_trace_plan: the choice timed on the first call of the size
    class, else the size rule).  The paths: one CTA (1 kernel); reduce / carry
    / apply (5 kernels up to 8,192 variables, else 3); a reduce / carry / apply
    prefix, the stuck bitmap, the single-pass scan, final statuses and the
    first-fault merge (7); the epoch path (a sorted check of the first part --
    pairs, three kernels per radix pass, the segmented scan's reduce, carry
    and apply -- and the stuck
    bitmap, then per epoch the stream filter, block sums, chunk offsets,
    gather, the candidates' sorted check, the gated fallback scan's set-up,
    scan and final statuses, and the gated merge with bitmap rebuild); or the
    single-pass scan and the final statuses (2)."""
    import paper_1910_11110_gb300 as amc
    path, n = amc.trace_plan(n_ops, n_vars, has_init)
    return TRACE_PATH_TEXT[path], n


def scan_traffic(n_ops, n_vars):
    """DRAM bytes of one check: not measured at this size.  A capture of the
    2^30-op check would hold more memory on the device and run longer than a
    profiling capture may, and the check's kernels do not scale in proportion
    to the trace (the first part and the per-variable passes are fixed), so a
    smaller capture's bytes are not scaled up here: None."""
    return None

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in ("all", "trace"):
        run_ours(args)
    else:
        import torch

        import paper_1910_11110_gb300 as amc
        torch.cuda.set_device(0)
        amc.build()
        dev = torch.device("cuda", 0)
        fn = {"uniform": lambda: measure_uniform(args, amc, dev), "vectorpu": lambda: measure_vectorpu(args, amc, dev),
              "well_declared": lambda: measure_well_declared(args, amc, dev),
              "kloc": lambda: measure_kloc(args, amc, dev),
              "programs": lambda: measure_programs(args, amc, dev), "serve": lambda: measure_serve(args, amc, dev),
              "vectorpu_lifetimes": lambda: measure_lifetimes(args, amc, dev),
              "programs_guarded": lambda: measure_guarded(args, amc, dev),
              "trace_sizes": lambda: measure_sizes(args, amc, dev)}
        print(json.dumps(fn[args.workload]()), flush=True)


if __name__ == "__main__":
    main()
