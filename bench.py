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
import tempfile
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
    ap.add_argument("--e2e-chunk", type=int, default=0, help="ops per chunk of the host-buffer check (0: 2^25)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=25.0)
    ap.add_argument("--workload", default="trace", choices=["trace", "programs", "vectorpu", "serve"])
    ap.add_argument("--rates", default="1000,10000,100000")
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--n-progs", type=int, default=100_000, help="programs workload: number of programs")
    ap.add_argument("--no-plain", action="store_true", help="programs workload: skip the one-launch-per-program run")
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
                             "kernel": trace_kernels(n_ops, n_vars)[0], "kernel_ms": k_ms,
                             "algorithmic_bytes": alg_bytes},
                "gpu_launches": trace_kernels(n_ops, n_vars)[1] * args.steps,
                "clocks": clk, "e2e": e2e, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


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


def base_line(args, value, ms, config, **extra):
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic", "config": config}
    line.update(extra)
    return line


def run_programs(args):
    """Batched persistent launch (graph replay) vs one launch per program."""
    import numpy as np
    import torch

    import paper_1910_11110_gb300 as amc
    import workloads
    torch.cuda.set_device(0)
    amc.build()
    b = workloads.programs(n_progs=args.n_progs)
    dev = torch.device("cuda")
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    tok, pay, off, nv = t(b["tok"]), t(b["payload"]), t(b["prog_tok_off"]), t(b["prog_nvars"])
    vo = torch.zeros(nv.numel() + 1, dtype=torch.int64, device=dev)
    torch.cumsum(nv.to(torch.int64), 0, out=vo[1:])
    n_tok = tok.numel()
    P = nv.numel()
    out = dict(step_mask=torch.empty(n_tok, dtype=torch.uint8, device=dev),
               final_mask=torch.empty(int(vo[-1]), dtype=torch.uint8, device=dev),
               prog_first_fault=torch.empty(P, dtype=torch.int64, device=dev))
    stream = torch.cuda.Stream()
    ws = torch.empty(amc.lib().amc_check_batch_workspace(n_tok, P, int(vo[-1])) + 256, dtype=torch.uint8, device=dev)
    ws = ws[(-ws.data_ptr()) % 256:]
    with torch.cuda.stream(stream):
        batched = lambda: amc.check_batch(tok, pay, off, nv, vo, graph_capture=True, out=out, workspace=ws,
                                          stream=stream)
        for _ in range(max(3, args.warmup)):
            batched()
        assert amc.sync_status(stream) == 0
        ms_b = timed(batched, args.steps, stream)
        # plain: one launch per program through the same entry point (no graph)
        offs = b["prog_tok_off"]
        L = amc.lib()
        import ctypes
        sp = ctypes.c_void_p(stream.cuda_stream)
        P_ = lambda x: ctypes.c_void_p(x)

        def plain():
            # one launch per program: the CSR arrays are offset to the
            # program, token and mask buffers stay whole (absolute offsets)
            for i in range(P):
                L.amc_check_batch(P_(tok.data_ptr()), P_(pay.data_ptr()), P_(off.data_ptr() + 8 * i),
                                  P_(nv.data_ptr() + 4 * i), P_(vo.data_ptr() + 8 * i), 1, n_tok,
                                  P_(out["step_mask"].data_ptr()), P_(out["final_mask"].data_ptr()),
                                  P_(out["prog_first_fault"].data_ptr() + 8 * i), 0, P_(ws.data_ptr()), ws.numel(),
                                  sp)
        ms_p = None
        if not args.no_plain:
            plain()
            assert amc.sync_status(stream) == 0
            ms_p = timed(plain, 1, stream)
    leaf = int(b["n_leaf"].sum())
    line = base_line(args, n_tok / (ms_b * 1e-3), ms_b,
                     {"workload": "programs", "n_progs": P, "tokens": n_tok, "leaf_ops": leaf, "seed": 3,
                      "mode": "batched persistent launch, CUDA graph replay, longest-first queue"},
                     plain=None if ms_p is None else {"value": n_tok / (ms_p * 1e-3), "ms_per_step": ms_p,
                                                      "mode": "one launch per program, same kernel"},
                     batched_over_plain=None if ms_p is None else ms_p / ms_b, gpu_launches=args.steps * 4)
    print(json.dumps(line), flush=True)


def vectorpu_launches(n_statements, n_vars):
    """Kernels of one translation + guarded check: 11 for the translation
    (two overlap passes, count, emit, total, two 3-kernel scans), then per
    check pass the reduce / carry / apply path (traces over at most 16,384
    variables from 2^20 ops on: 5 kernels up to 8,192 variables -- warp
    batches and a two-level carry -- else 3), or the scan kernel plus, in the
    second pass, the final-status kernel."""
    if n_vars <= 16384 and n_statements >= (1 << 20) and os.environ.get("AMC_SCAN_DENSE", "") != "0":
        return 11 + 2 * (5 if n_vars <= 8192 else 3)
    return 11 + 1 + 2


def run_vectorpu(args):
    """Translation + guarded check of the 2^24-call VectorPU workload."""
    import numpy as np
    import torch

    import paper_1910_11110_gb300 as amc
    import workloads
    torch.cuda.set_device(0)
    amc.build()
    w = workloads.vectorpu_calls(seed=2)
    dev = torch.device("cuda")
    d = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in w.items()}
    A = d["arr_start"].numel()
    stream = torch.cuda.current_stream()
    tr = amc.translate_vectorpu(d["arr_start"], d["arr_len"], d["call_side"], d["call_off"], d["opnd_array"],
                                d["opnd_mode"])
    n = tr["n"]
    cap = n
    res = {}

    def step():
        r = amc.translate_vectorpu(d["arr_start"], d["arr_len"], d["call_side"], d["call_off"], d["opnd_array"],
                                   d["opnd_mode"], out_cap=cap)
        res["o"] = amc.check_trace(r["kind_side"], r["var"], 2 * A, guarded=True)

    for _ in range(max(3, args.warmup)):
        step()
    assert amc.sync_status() == 0
    ms = timed(step, args.steps, stream)
    n_calls = d["call_side"].numel()
    line = base_line(args, n / (ms * 1e-3), ms,
                     {"workload": "vectorpu_calls", "n_arrays": A, "n_calls": n_calls, "statements": n, "seed": 2},
                     calls_per_s=n_calls / (ms * 1e-3), gpu_launches=args.steps * vectorpu_launches(n, 2 * A))
    print(json.dumps(line), flush=True)


def run_serve(args):
    """Open-loop Poisson arrivals into the continuous-batching server."""
    import threading

    import numpy as np
    import torch

    import paper_1910_11110_gb300 as amc
    import workloads
    torch.cuda.set_device(0)
    amc.build()
    rng = np.random.default_rng(4)
    pool_n = 1 << 25
    pool_ks = ((rng.choice(5, size=pool_n, p=workloads.KIND_MIX)) | (rng.integers(0, 2, pool_n) << 4)).astype(np.uint8)
    pool_var = rng.integers(0, 1 << 30, pool_n).astype(np.int64)
    results = {}
    for rate in [float(x) for x in args.rates.split(",")]:
        n_req = args.serve_requests
        arr = np.cumsum(rng.exponential(1.0 / rate, n_req))
        # sessions of 1..64 requests over 64..4096 vars, typed by kind
        sess = []
        while sum(x[1] for x in sess) < n_req:
            sess.append((len(sess), int(rng.integers(1, 65)), int(rng.integers(64, 4097)), int(rng.integers(0, 2))))
        order = np.repeat(np.arange(len(sess)), [x[1] for x in sess])[:n_req]
        rng.shuffle(order)
        reqs = []
        for k, si in enumerate(order):
            sid, _, nv, kind = sess[si]
            if kind == 0:
                n = int(2 ** rng.uniform(10, 24))
                a = int(rng.integers(0, pool_n - n))
                reqs.append((sid, kind, nv, ("trace", a, n)))
            else:
                reqs.append((sid, kind, nv, ("prog", k)))
        with amc.Server(mem_budget_bytes=32 << 30, max_slots=32) as srv:
            tickets = {}
            lat = []
            ops = [0]
            done_flag = [False]

            def poller():
                while not done_flag[0] or tickets:
                    for t in list(tickets):
                        r = srv.poll(t)
                        if r is not None:
                            lat.append(r["t_done"] - r["t_submit"])
                            ops[0] += len(r["status"])
                            tickets.pop(t)
                    time.sleep(2e-5)

            th = threading.Thread(target=poller)
            th.start()
            t0 = time.perf_counter()
            for (sid, kind, nv, spec), at in zip(reqs, arr):
                while time.perf_counter() - t0 < at:
                    pass
                if spec[0] == "trace":
                    _, a, n = spec
                    ks = pool_ks[a:a + n]
                    var = (pool_var[a:a + n] % nv).astype(np.int32)
                else:
                    b = workloads.programs(1, seed=44, first=spec[1], vars_lo=nv, vars_hi=nv)
                    ks, var = b["tok"], b["payload"]
                while (t := srv.submit(sid, kind, nv, ks, var)) is None:
                    time.sleep(1e-4)
                tickets[t] = 1
            done_flag[0] = True
            th.join()
            wall = time.perf_counter() - t0
        lat = np.array(lat) * 1e3
        results[str(int(rate))] = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                                   "ops_per_s": ops[0] / wall, "requests": n_req, "wall_s": wall}
    first = results[list(results)[0]]
    line = base_line(args, first["ops_per_s"], None,
                     {"workload": "serve", "rates_req_per_s": args.rates, "requests_per_rate": args.serve_requests,
                      "slots": 32, "budget_gb": 32, "seed": 4},
                     serve=results)
    print(json.dumps(line), flush=True)


def tail_epochs(n_ops):
    """Epochs of the long-trace path at its default shape (first part 2^22
    ops, each epoch ending at four times its start)."""
    e0, k = 1 << 22, 0
    while e0 < n_ops:
        e0, k = min(e0 << 2, n_ops), k + 1
    return k


def trace_kernels(n_ops, n_vars):
    """(what the timed span covers, kernels launched per check) for
    amc_check_trace without initial statuses: the reduce / carry / apply path
    over at most 16,384 variables from 2^20 ops; over more (at most 2^20)
    variables from 2^24 ops that path on the first 2^22 ops, then the stuck
    bitmap seeded from its final statuses, the single-pass scan, the final
    statuses and the first-fault merge (7 kernels); from 2^29 ops the first
    2^22 ops as pairs sorted by variable (pairs, 3 radix passes of histogram,
    scan and scatter, then the single-pass segmented scan: 11 kernels), then
    per epoch the stuck bitmap, stream filter, block sums, chunk offsets,
    gather, the candidates' sorted check (10), the gated fallback scan
    (set-up, scan, final statuses) and the gated first-fault merge (19
    kernels); else the scan and the final statuses."""
    if os.environ.get("AMC_SCAN_DENSE", "") == "0":
        return "scan_trace_kernel", 2
    if n_vars <= 8192 and n_ops >= (1 << 20):
        return "warp reduce + carry + apply kernels", 5
    if n_vars <= 16384 and n_ops >= (1 << 20):
        return "dense reduce + carry + apply kernels", 3
    if 16384 < n_vars <= (1 << 20) and n_ops >= (1 << 29) and os.environ.get("AMC_SCAN_TAIL", "") != "0":
        return ("first 2^22 ops: sorted check (radix sort by variable + segmented scan); epochs to 4x their "
                "start: tail_filter_kernel + gather + sorted check of the candidates"), 11 + 19 * tail_epochs(n_ops)
    if 16384 < n_vars <= (1 << 20) and n_ops >= (1 << 24):
        return "prefix (dense reduce + carry + apply) + scan_trace_kernel", 7
    return "scan_trace_kernel", 2


def scan_traffic(n_ops, n_vars):
    """DRAM bytes (read + write) of one check -- every kernel of the timed span
    -- from the recorded ncu capture, or None when the capture was of another
    workload or the kernel sources have changed since (the record keeps the
    SHA-256 of scan_trace.cu, scan_dense.cu, scan_tail.cu and scan_sorted.cu)."""
    import hashlib
    tr_path = os.path.join(ROOT, "profiles", "scan_trace_zipf_traffic.json")
    h = hashlib.sha256()
    try:
        rec = json.load(open(tr_path))
        for f in ("scan_trace.cu", "scan_dense.cu", "scan_tail.cu", "scan_sorted.cu"):
            h.update(open(os.path.join(ROOT, "paper_1910_11110_gb300", "csrc", f), "rb").read())
        sha = h.hexdigest()
    except Exception:
        return None
    if rec.get("source_sha256") != sha or rec.get("n_ops") != n_ops or rec.get("n_vars") != n_vars:
        return None
    return rec.get("bytes_per_launch")


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "programs":
        run_programs(args)
    elif args.workload == "vectorpu":
        run_vectorpu(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
