#!/usr/bin/env python3
"""Benchmark of the GB300 access-mode consistency checker.

One step = one amc_check_trace call over the 2^30-op, 2^20-variable Zipf(1.05)
trace (kind mix r .40 / w .20 / Push .15 / Pull .15 / Noop .10, fair side,
seed 1): every per-step status, final status and first fault.  Inputs (5.4 GB)
are resident in HBM when the timed region starts and exceed L2, so no L2 flush
is needed between steps.

Prints one JSON line (rank 0).  Under torchrun (N > 1) each rank checks its own
replica of the trace on its own GPU ("replicas only": the path has no exchange
step); value = ops of all ranks / max time over ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--n-ops N] [--n-vars V] [--no-e2e] [--no-cpu]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

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
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
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
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{gpu_index}.csv")

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


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


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
    m = int(min(len(ks_host), max(n, n * budget_s / max(dt, 1e-6))))
    t0 = time.perf_counter()
    oracle.check_trace(ks_host[:m], var_host[:m], n_vars)
    dt = time.perf_counter() - t0
    return {"value": m / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {m} ops of the same trace, one pass, single thread ({dt:.1f} s)"}


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
    stream = torch.cuda.current_stream()

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
    ms_total = max_over_ranks(ms_total, world)
    ms_step = ms_total / args.steps
    k_ms = statistics.mean(a.elapsed_time(b) for a, b in zip(k_start, k_stop))
    value = n_ops * world / (ms_step * 1e-3)

    peak, peak_kind = peaks()
    alg_bytes = 6 * n_ops + 5 * n_vars
    achieved = alg_bytes / (k_ms * 1e-3) / 1e9
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "scan_trace_zipf_traffic.json")
    if os.path.exists(tr_path):
        try:
            traffic = json.load(open(tr_path)).get("bytes_per_launch")
        except Exception:
            traffic = None

    # end-to-end through the public API: pinned host inputs, H2D, check, D2H
    e2e = None
    if not args.no_e2e:
        ks_h = torch.empty(n_ops, dtype=torch.uint8, pin_memory=True)
        var_h = torch.empty(n_ops, dtype=torch.int32, pin_memory=True)
        ks_h.copy_(ks)
        var_h.copy_(var)
        step_h = torch.empty(n_ops, dtype=torch.uint8, pin_memory=True)
        fin_h = torch.empty(n_vars, dtype=torch.uint8, pin_memory=True)
        vff_h = torch.empty(n_vars, dtype=torch.int32, pin_memory=True)
        ff_h = torch.empty(1, dtype=torch.int64, pin_memory=True)
        ks_d = torch.empty_like(ks)
        var_d = torch.empty_like(var)

        def e2e_step():
            ks_d.copy_(ks_h, non_blocking=True)
            var_d.copy_(var_h, non_blocking=True)
            amc.check_trace(ks_d, var_d, n_vars, out=out, workspace=ws, stream=stream)
            step_h.copy_(out["step_status"], non_blocking=True)
            fin_h.copy_(out["final_status"], non_blocking=True)
            vff_h.copy_(out["var_first_fault"], non_blocking=True)
            ff_h.copy_(out["first_fault"], non_blocking=True)

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
               "ms_per_step": e_ms}
        if amc.sync_status() != 0:
            raise RuntimeError("device error during e2e steps")
        host_copy = (ks_h.numpy(), var_h.numpy())
    else:
        host_copy = None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        if host_copy is None:
            m = 1 << 26
            host_copy = (ks[:m].cpu().numpy(), var[:m].cpu().numpy())
        cpu = cpu_baseline(host_copy[0], host_copy[1], n_vars, args.cpu_seconds)

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
                             "kernel": "scan_trace_kernel", "kernel_ms": k_ms,
                             "algorithmic_bytes": alg_bytes},
                "gpu_launches": 2 * args.steps,
                "clocks": clk, "e2e": e2e, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def ctypes_ptr(ev):
    import ctypes
    return ctypes.c_void_p(ev.cuda_event)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
