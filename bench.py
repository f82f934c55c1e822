#!/usr/bin/env python3
"""Benchmark of the GB300 CoS evaluator (edge.sample updates/s).

One step = one pass of the hot path over one batch of synthetic samples:
attach the samples (device-resident times, transposed on the GPU) and evaluate
the path sums of every sample (propagator table, level walk, sink values,
compensated mean) through the C ABI.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload large|medium|tiny|batched|serving]
                  [--impl ours|reference]

The default workload is the large graph (2^20 samples per GPU, FP32 bulk / FP64
sink), the largest configuration that fits one GPU.  With --gpus N > 1 and no
torchrun environment, the script starts N local ranks itself (torch.distributed.run
on 127.0.0.1); every rank evaluates its own batch of samples of the same graph
(weak scaling, no data-path collective) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from workloads import large, medium, tiny  # noqa: E402

WORKLOADS = {
    # name: (factory, mode name, description)
    "medium": (medium, "fp64", "medium leveled DAG: L=10, widths 1..4096..1, N=18498, E=46188, fan-in U{1..4}, "
                               "K=16 kinds, D=10 times, 65536 samples per GPU, beta=10, plain FP64"),
    "large": (large, "mixed", "large leveled DAG: L=14, widths 1..262144..1, N=2105474, E=5263492, geometric "
                              "fan-in 1..6, K=32, D=14, 2^20 samples per GPU, FP32 bulk / FP64 sink"),
    "tiny": (tiny, "fp64", "tiny leveled DAG: L=6, widths [1,4,8,8,4,1], N=26, K=4, D=6, 1024 samples, FP64"),
}
MODES = {"fp64": 0, "mixed": 1, "count": 2}
DTYPE = {"fp64": "f64", "mixed": "f32 (sink and sample sums f64)", "count": "int64"}
L2_FLUSH_BYTES = 512 << 20
FALLBACK_HBM_GBS = 6800.0
# Nominal FP64 multiply-add issue rate of GB300 per SM and clock (1.25 TFLOP/s over
# 152 SMs at 2070 MHz); used only if the live probe (cos_probe_fma_rate) fails.
NOMINAL_DFMA_PER_CLK_SM = 2.0
# A step longer than this is timed end to end (e2e) on at most E2E_LONG_STEPS steps.
E2E_LONG_STEP_S = 0.5
E2E_LONG_STEPS = 5
# Oracle check of the timed run's results: every sample up to this many, else the
# first ORACLE_SLICE samples (a contiguous slice), plus a few for the long-double reference.
ORACLE_FULL_MAX = 1 << 17
ORACLE_SLICE = 1024
ORACLE_TIGHT = 64
BATCH_CHECK_SAMPLES = 32          # batched workload: samples of every graph compared with the oracle
SERVING_CHECK_REQUESTS = 8        # serving: completed requests per form whose means meet the oracle


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["serving", "batched"], default="large")
    ap.add_argument("--num-graphs", type=int, default=64, help="batched: graphs in the launch")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: Poisson arrival rate (requests/s)")
    ap.add_argument("--duration", type=float, default=60.0, help="serving: seconds of arrivals")
    ap.add_argument("--pool-size", type=int, default=128, help="serving: resident graphs")
    ap.add_argument("--max-nodes", type=float, default=2e6, help="serving: largest graph")
    ap.add_argument("--max-queue", type=int, default=256, help="serving: bounded wait queue (excess is shed)")
    ap.add_argument("--budget-gb", type=float, default=150.0, help="serving: device memory budget")
    ap.add_argument("--sweep-rates", type=str, default="", help="serving: extra sustainable rates, e.g. 4,8")
    ap.add_argument("--sweep-duration", type=float, default=30.0, help="serving: seconds per extra rate")
    ap.add_argument("--serving-forms", type=str, default="resident,batched,plain",
                    help="serving: forms to run (resident, batched, plain)")
    ap.add_argument("--inflight-work", type=float, default=None,
                    help="serving: resident server's cap on held work (edge x samples)")
    ap.add_argument("--inflight-max", type=int, default=None, help="serving: resident server's cap on held requests")
    ap.add_argument("--mode", choices=sorted(MODES), default=None)
    ap.add_argument("--abs", action="store_true",
                    help="the same walk also sums |path| values (COS_EVAL_ABS; fp64 and mixed modes)")
    ap.add_argument("--samples", type=int, default=None, help="samples per GPU (default: the workload's)")
    ap.add_argument("--tuning", type=str, default="", help="JSON dict passed to cos_set_tuning")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the launch shape with cos_autotune on the workload before timing")
    ap.add_argument("--cpu-baseline-seconds", type=float, default=15.0)
    ap.add_argument("--reference-seconds", type=float, default=120.0,
                    help="reference arm: about how long its warm-up and timed steps take in total")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true")
    return ap.parse_args(argv)


# ------------------------------------------------------------------ distributed plumbing

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seed(base_seed: int, rank: int) -> int:
    """Rank 0 uses the workload's own seed; rank r > 0 draws its own samples."""
    return base_seed if rank == 0 else base_seed * 1000003 + rank


def max_over_ranks(value: float, world: int, device=None) -> float:
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def combine_means(local_sum: float, local_count: int, world: int, device=None) -> float:
    """The one exchange of the sample-sharded path: every rank's sample sum and count
    summed over ranks (FP64 all-reduce), giving the mean over all ranks' samples."""
    if world <= 1:
        return local_sum / max(local_count, 1)
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_sum, float(local_count)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t[0].item()) / max(float(t[1].item()), 1.0)


def free_port() -> int:
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def launch_ranks(n: int, argv) -> int:
    """Start n local ranks of this script (one per GPU) under torch.distributed.run on
    127.0.0.1 and return their exit status; rank 0 prints the JSON line."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), os.path.abspath(__file__)] + list(argv)
    return subprocess.call(cmd)


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""
    QUERY = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 10:
                    continue
                if self.uuid and parts[1] != self.uuid:
                    continue
                try:
                    rows.append((float(parts[2]), float(parts[3]), parts[6:10]))
                except ValueError:
                    continue
        os.unlink(self.path)
        if not rows:
            return None
        seen = sorted({name for _, _, flags in rows for name, fl in zip(self.REASONS, flags) if fl == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": seen, "samples": len(rows)}


# ------------------------------------------------------------------ measured peaks and profiles

def fp64_fma_peak(cg, dev_index: int):
    """FP64 multiply-add peak in TFLOP/s (2 flops per FMA): measured live by the probe
    kernel, else the nominal issue rate x SMs x the measured maximum SM clock."""
    import torch
    try:
        return 2.0 * cg.probe_fma_rate(0) / 1e12, "measured: FP64 FMA probe kernel (cos_probe_fma_rate) on this GPU"
    except Exception:
        sms = torch.cuda.get_device_properties(dev_index).multi_processor_count
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                mhz = float(json.load(f)["sm_max_mhz"])
        except (OSError, KeyError, ValueError):
            mhz = 2070.0
        return (2.0 * NOMINAL_DFMA_PER_CLK_SM * sms * mhz * 1e6 / 1e12,
                f"nominal: {sms} SMs x {NOMINAL_DFMA_PER_CLK_SM:g} DFMA/clk x {mhz:g} MHz")


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def profiled_traffic(kernel_tag: str, samples: int, schedule: int, layout: int):
    """DRAM bytes per launch from the committed ncu summary, if it covers this kernel build,
    schedule and layout.  The walk's traffic grows in proportion to the samples (per-sample
    slabs, per-chunk items), so the profiled figure is scaled to this launch's sample count."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            v = json.load(f).get(kernel_tag)
    except (OSError, ValueError):
        return None
    if not isinstance(v, dict) or v.get("schedule") != schedule or v.get("layout") != layout:
        return None
    return v["bytes_per_launch"] * samples / v["samples"]


# ------------------------------------------------------------------ CPU oracle timing

def oracle_rate(graph, samples, seconds: float, nthreads: int = 0):
    """Edge.sample updates/s of the CPU oracle on a bounded prefix of the samples, sized
    from a short timed run after a warm-up (thread pool start, first touch)."""
    import oracle
    oracle.build()
    n = 32
    oracle.evaluate(graph, samples.eps, samples.beta, samples.t[:n], with_abs=False, nthreads=nthreads)
    t0 = time.perf_counter()
    oracle.evaluate(graph, samples.eps, samples.beta, samples.t[:n], with_abs=False, nthreads=nthreads)
    dt = time.perf_counter() - t0
    n2 = int(min(samples.num_samples, max(n, n * seconds / max(dt, 1e-6))))
    t0 = time.perf_counter()
    oracle.evaluate(graph, samples.eps, samples.beta, samples.t[:n2], with_abs=False, nthreads=nthreads)
    dt = time.perf_counter() - t0
    return graph.num_edges * n2 / dt, n2, dt


# ------------------------------------------------------------------ our arm

def run_ours(args, rank, world, local):
    import torch
    import paper_2501_00675_gb300 as cg
    from paper_2501_00675_gb300 import _build

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    factory, default_mode, desc = WORKLOADS[args.workload]
    mode_name = args.mode or default_mode
    mode = MODES[mode_name]
    if args.abs and mode == 2:
        raise SystemExit("--abs needs a floating-point mode")
    emode = mode | (cg.COS_EVAL_ABS if args.abs else 0)     # the mode argument of cos_evaluate
    nout = 2 if args.abs else 1                              # per-sample outputs: R, then A
    kw = {} if args.samples is None else {"num_samples": args.samples}
    base = factory(**kw)
    wl = factory(seed=rank_seed({"medium": 1, "large": 2, "tiny": 0}[args.workload], rank), **kw) if rank else base
    # the graph is the workload's (replicated on every rank); samples are per rank
    g, s = base.graph, wl.samples
    S, E, N, D, K = s.num_samples, g.num_edges, g.num_nodes, g.num_times, g.num_kinds

    if not os.path.exists(_build.LIB):
        _build.build()
    cg.load_library()
    gr = cg.Graph.from_workload_graph(g)
    if args.tuning:
        gr.set_tuning(**json.loads(args.tuning))
    stream = torch.cuda.current_stream(dev)
    t_dev = torch.from_numpy(s.t).to(dev)                                   # [S][D], resident in HBM
    out_dtype = torch.int64 if mode == 2 else torch.float64
    out = torch.empty(nout * S, dtype=out_dtype, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step():
        gr.set_samples(t_dev, s.eps, s.beta, cg.COS_T_SAMPLE_MAJOR, stream=stream)
        gr.evaluate(emode, out=out, want_mean=False, stream=stream, allow_overflow=True)

    if args.autotune:
        step()
        gr.autotune(emode, out=out, stream=stream)   # times candidate shapes on these samples, keeps the fastest
    for _ in range(args.warmup):
        step()
    gr.get_result(stream)
    torch.cuda.synchronize()
    tuning = gr.get_tuning(emode)

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid).start()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()                                                       # untimed L2 flush
        ev[k][0].record(stream)
        gr.set_samples(t_dev, s.eps, s.beta, cg.COS_T_SAMPLE_MAJOR, stream=stream)
        ev[k][1].record(stream)
        gr.evaluate(emode, out=out, want_mean=False, stream=stream, allow_overflow=True)
        ev[k][2].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    mean = gr.get_result(stream) if mode != 2 else float("nan")
    mean_all = combine_means(mean * S, S, world, dev) if mode != 2 else float("nan")   # untimed
    step_ms = [ev[k][0].elapsed_time(ev[k][2]) for k in range(args.steps)]
    walk_ms = [ev[k][1].elapsed_time(ev[k][2]) for k in range(args.steps)]
    total_s = sum(step_ms) / 1e3
    total_s = max_over_ranks(total_s, world, dev)
    units = float(E) * S * args.steps * world
    value = units / total_s

    # roofline of the walker kernel (one launch per evaluate)
    w_bytes = 4 if mode == 1 else 8
    alg_bytes = S * (2.0 * N * w_bytes + D * 8 + 8)
    if args.abs:                                                        # A's float node values and result
        alg_bytes += S * (2.0 * N * 4 + 8)
    walk_s = statistics.mean(walk_ms) / 1e3
    peak, peak_kind = hbm_peak()
    hbm = {"bound": "hbm", "achieved": alg_bytes / walk_s / 1e9, "peak": peak, "unit": "GB/s",
           "frac": alg_bytes / walk_s / 1e9 / peak, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
           if peak_kind == "measured" else "fallback 6.8 TB/s",
           "traffic": profiled_traffic(f"walk_{mode_name}{'_abs' if args.abs else ''}_{args.workload}",
                                       S, tuning["schedule"], tuning["layout"]),
           "algorithmic_bytes_per_launch": alg_bytes}
    if mode == 0:
        tflops = 2.0 * E * S / walk_s / 1e12
        fp64_peak, fp64_src = fp64_fma_peak(cg, local)
        alu = {"bound": "alu", "achieved": tflops, "peak": fp64_peak, "unit": "TFLOP/s",
               "frac": tflops / fp64_peak, "peak_source": fp64_src,
               "traffic": hbm["traffic"], "algorithmic_flops_per_launch": 2.0 * E * S}
        roofline, other = (alu, hbm) if alu["frac"] >= hbm["frac"] else (hbm, alu)
    else:
        roofline, other = hbm, None

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        t_host = torch.from_numpy(s.t).pin_memory()
        r_host = torch.empty(nout * S, dtype=out_dtype).pin_memory()
        for _ in range(2):
            gr.set_samples(t_host, s.eps, s.beta, cg.COS_T_HOST | cg.COS_T_SAMPLE_MAJOR, stream=stream)
            gr.evaluate(emode, out=out, want_mean=False, stream=stream, allow_overflow=True)
            r_host.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
        e_ms = []
        e2e_steps = args.steps if total_s / args.steps <= E2E_LONG_STEP_S else min(args.steps, E2E_LONG_STEPS)
        barrier(world)
        for k in range(e2e_steps):
            flush.zero_()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            gr.set_samples(t_host, s.eps, s.beta, cg.COS_T_HOST | cg.COS_T_SAMPLE_MAJOR, stream=stream)
            gr.evaluate(emode, out=out, want_mean=False, stream=stream, allow_overflow=True)
            r_host.copy_(out, non_blocking=True)
            b.record(stream)
            b.synchronize()
            e_ms.append(a.elapsed_time(b))
        barrier(world)
        e_total = max_over_ranks(sum(e_ms) / 1e3, world, dev)
        e2e = {"value": float(E) * S * e2e_steps * world / e_total, "unit": "edge·sample updates/s",
               "h2d_bytes_per_step": int(S * D * 8 + K * 8), "d2h_bytes_per_step": int(nout * S * 8),
               "steps": e2e_steps}

    # error of the timed run's results against the FP64 oracle, relative to sum |paths|
    err = None
    if rank == 0 and not args.no_oracle_check:
        import oracle
        full = S <= ORACLE_FULL_MAX
        n_chk = S if full else min(S, ORACLE_SLICE)      # every sample, or the first ORACLE_SLICE
        out_all = out.cpu().numpy()
        got_all = out_all[:S]
        got = got_all[:n_chk]
        if mode == 2:
            cnt, _ = oracle.count_paths(g)
            err = {"bit_exact": bool(np.all(got_all == cnt)), "samples_checked": int(S)}
        else:
            t0 = time.perf_counter()
            R_or, A_or = oracle.evaluate(g, s.eps, s.beta, s.t[:n_chk])
            oracle_s = time.perf_counter() - t0
            rel = np.abs(got - R_or) / A_or
            tol = 1e-12 if mode == 0 else 1e-5
            err = {"max_err_over_abs_path_sum": float(rel.max()) if n_chk else 0.0,
                   "median_err_over_abs_path_sum": float(np.median(rel)) if n_chk else 0.0,
                   "tolerance": tol, "samples_checked": int(n_chk),
                   "samples": "all" if full else f"the first {n_chk} (contiguous)", "oracle_s": oracle_s,
                   "within_tolerance": bool(np.all(np.abs(got - R_or) <= tol * A_or))}
            if full and S:
                # the timed run's compensated mean against the oracle's Neumaier mean of all samples
                err["mean_err_over_mean_abs_path_sum"] = float(abs(mean - oracle.neumaier_mean(R_or)) / np.mean(A_or))
            if args.abs and n_chk:                                        # A(s) from the same walk
                err["abs_max_rel_err"] = float(np.max(np.abs(out_all[S:S + n_chk] - A_or) / A_or))
            nt = min(n_chk, ORACLE_TIGHT)                  # long-double reference on a few samples
            R_ld = oracle.evaluate_tight(g, s.eps, s.beta, s.t[:nt])
            err["max_err_vs_long_double"] = float((np.abs(got[:nt] - R_ld) / A_or[:nt]).max()) if nt else 0.0
            err["oracle_max_err_vs_long_double"] = float((np.abs(R_or[:nt] - R_ld) / A_or[:nt]).max()) if nt else 0.0
            err["long_double_samples"] = int(nt)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, n, dt = oracle_rate(g, s, args.cpu_baseline_seconds)
        cpu = {"value": rate, "unit": "edge·sample updates/s", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
               "sample": f"first {n} of {S} samples of the same workload ({dt:.1f} s, OpenMP over samples)"}
    gr.close()
    if rank != 0:
        return None
    line = {
        "metric": "edge·sample updates/s", "value": value, "unit": "edge·sample updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[mode_name],
        "data": "synthetic (seeded random leveled DAG and uniform sample times)",
        "config": {"workload": desc, "mode": mode_name + ("+abs" if args.abs else ""), "samples_per_gpu": S, "graph": {"L": g.num_levels, "N": N, "E": E,
                   "K": K, "D": D}, "parallelism": f"sample-sharded x{world}, graph replicated, no collective",
                   "l2": "flushed between timed steps (512 MB write); working set larger than L2",
                   "tuning": tuning},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 2 * args.steps,
        "clocks": clk, "walk_ms_per_launch": statistics.mean(walk_ms), "mean_R": mean, "mean_R_all_ranks": mean_all, "error_vs_oracle": err,
    }
    if other is not None:
        line["roofline_secondary"] = other
    return line


# ------------------------------------------------------------------ batched uneven

def run_batched(args, rank, world, local):
    """64 graphs of uneven order and sample count in one persistent, CUDA-graph-captured
    launch (mixed mode), launch shape picked by the autotuner on a capped-sample copy;
    compared with the same graphs evaluated one after another."""
    import torch
    import paper_2501_00675_gb300 as cg
    from workloads import batched

    torch.cuda.set_device(local)
    cg.load_library(build_if_missing=True)
    mode = MODES[args.mode or "mixed"]
    t0 = time.perf_counter()
    wls = batched(seed=3 + 1000 * rank, num_graphs=args.num_graphs)
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    graphs, outs, probe = [], [], []
    for w in wls:
        g = cg.Graph.from_workload_graph(w.graph)
        inf = g.info()
        psb = 2 * 8 * inf["W_max"] + 8 * inf["P"]          # workspace bytes per sample of a tile
        g.set_tuning(tile_samples=int(max(128, min(65536, (2 << 30) // psb // 128 * 128))))   # <= 2 GB per graph
        g.set_samples(torch.from_numpy(w.samples.t).cuda(), w.samples.eps, w.samples.beta, cg.COS_T_SAMPLE_MAJOR)
        graphs.append(g)
        outs.append(torch.empty(w.samples.num_samples, dtype=torch.float64, device="cuda"))
        cap = min(w.samples.num_samples, 16384)
        h = g.share()
        h.set_tuning(tile_samples=min(16384, g.get_tuning(mode)["tile_samples"]))
        h.set_samples(torch.from_numpy(w.samples.t[:cap].copy()).cuda(), w.samples.eps, w.samples.beta,
                      cg.COS_T_SAMPLE_MAJOR)
        probe.append(h)
    units = float(sum(w.graph.num_edges * w.samples.num_samples for w in wls))
    tb = cg.Batch(probe, mode)
    best = tb.autotune()
    tb.close()
    for h in probe:
        h.close()
    b = cg.Batch(graphs, mode, outs)
    b.set_tuning(samples_per_lane=best["samples_per_lane"], rows_per_warp=best["rows_per_warp"], layout=best["layout"])
    for _ in range(max(args.warmup, 2)):           # second launch captures the CUDA graph
        b.launch(stream)
    b.results(stream)
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):                     # every step's working set (GBs of slabs) exceeds L2
        b.launch(stream)
    e1.record(stream)
    e1.synchronize()
    barrier(world)
    step_ms = max_over_ranks(e0.elapsed_time(e1) / 1e3, world, local) * 1e3 / max(args.steps, 1)
    b.results(stream)
    # the timed launch's first samples of every graph, kept for the oracle check below
    n_chk = BATCH_CHECK_SAMPLES
    got = [o[:min(n_chk, w.samples.num_samples)].cpu().numpy() for o, w in zip(outs, wls)]
    # the same graphs one after another through cos_evaluate, same launch shape
    seq = []
    for g in graphs:
        g.set_tuning(samples_per_lane=best["samples_per_lane"], rows_per_warp=best["rows_per_warp"],
                     layout=best["layout"])
    for rep in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for g, o in zip(graphs, outs):
            g.evaluate(mode, out=o, want_mean=False, stream=stream)
        e1.record(stream)
        e1.synchronize()
        seq.append(e0.elapsed_time(e1))
    b.close()
    for g in graphs:
        g.close()
    if rank != 0:
        return None
    err = None if args.no_oracle_check else batched_oracle_check(wls, got, mode)
    t_b = step_ms / 1e3
    w_bytes = 4 if mode == 1 else 8
    alg_bytes = float(sum(w.samples.num_samples * (2.0 * w.graph.num_nodes * w_bytes + 8 * w.graph.num_times + 8)
                          for w in wls))
    peak, peak_kind = hbm_peak()
    roofline = {"bound": "hbm", "achieved": alg_bytes / t_b / 1e9, "peak": peak, "unit": "GB/s",
                "frac": alg_bytes / t_b / 1e9 / peak, "traffic": None,
                "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback 6.8 TB/s",
                "algorithmic_bytes_per_launch": alg_bytes}
    return {
        "metric": "edge·sample updates/s", "value": units * world / t_b, "unit": "edge·sample updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.mode or "mixed"], "data": "synthetic",
        "config": {"workload": batched_desc(len(wls)), "autotuned": best, "generation_s": gen_s,
                   "edge_samples": units, "l2": "no flush: every step's working set is GBs of node values"},
        "roofline": roofline, "gpu_launches": args.steps,
        "sequential_ms": min(seq), "batched_speedup_vs_sequential": min(seq) / step_ms,
        "error_vs_oracle": err,
    }


# ------------------------------------------------------------------ serving

def batched_oracle_check(wls, got, mode):
    """Every graph's first samples of the timed batched launch (got[g], host arrays)
    against the FP64 oracle on the same samples, relative to sum |paths| (bit-exact
    path counts in count mode)."""
    import oracle
    t0 = time.perf_counter()
    worst, ok, n_tot = 0.0, True, 0
    tol = 1e-12 if mode == 0 else 1e-5
    for w, r in zip(wls, got):
        n = r.size
        n_tot += n
        if mode == 2:
            cnt, _ = oracle.count_paths(w.graph)
            ok = ok and bool(np.all(r == cnt))
            continue
        R_or, A_or = oracle.evaluate(w.graph, w.samples.eps, w.samples.beta, w.samples.t[:n])
        if n:
            worst = max(worst, float(np.max(np.abs(r - R_or) / A_or)))
        ok = ok and bool(np.all(np.abs(r - R_or) <= tol * A_or))
    err = {"samples_checked": n_tot, "samples": f"the first {max((r.size for r in got), default=0)} of each "
                                                f"of the {len(wls)} graphs", "oracle_s": time.perf_counter() - t0}
    if mode == 2:
        err["bit_exact"] = ok
    else:
        err.update(max_err_over_abs_path_sum=worst, tolerance=tol, within_tolerance=ok)
    return err


def serving_oracle_check(torch, reqs, wpool, beta, mode, counter, n_req=SERVING_CHECK_REQUESTS):
    """Means of completed requests against the FP64 oracle: the n_req completed requests
    with the least work (edges x samples), their sample times drawn again from their
    seeds (the counter-based generator the resident kernel uses, or the seeded device
    generator of the batched server), the oracle's Neumaier mean compared with the
    served mean relative to the mean of sum |paths|."""
    import oracle
    from paper_2501_00675_gb300.serve import request_times
    from workloads import counter_times
    done = [r for r in reqs if r.status == "done" and r.spec.num_samples > 0]
    done.sort(key=lambda r: wpool[r.spec.graph_id][0].num_edges * r.spec.num_samples)
    worst, ok, t0 = 0.0, True, time.perf_counter()
    tol = 1e-12 if mode == 0 else 1e-5
    for r in done[:n_req]:
        g, eps = wpool[r.spec.graph_id]
        S, D = r.spec.num_samples, g.num_times
        if counter:
            t = counter_times(r.spec.seed, 0, S, D, beta)
        else:
            t = np.ascontiguousarray(request_times(torch, r.spec, D, beta)[:, :S].cpu().numpy().T)
        R, A = oracle.evaluate(g, eps, beta, t)
        e = abs(r.mean - oracle.neumaier_mean(R)) / float(np.mean(A))
        worst = max(worst, e)
        ok = ok and e <= tol
    return {"requests_checked": min(n_req, len(done)), "max_mean_err_over_mean_abs_path_sum": worst,
            "tolerance": tol, "within_tolerance": ok, "oracle_s": time.perf_counter() - t0}


def run_serving(args, rank, world, local):
    """Poisson request stream against the resident pool in the FP32/FP64-mixed mode:
    the resident server (the headline value), batched launches on two streams, and
    one-request-at-a-time plain FP64."""
    import torch
    import paper_2501_00675_gb300 as cg
    from paper_2501_00675_gb300.serve import RequestSpec, ResidentScheduler, Server, latency_summary, poisson_run
    from workloads import serving_pool

    torch.cuda.set_device(local)
    cg.load_library(build_if_missing=True)
    t0 = time.perf_counter()
    wpool = serving_pool(seed=4, pool_size=args.pool_size, max_nodes=args.max_nodes)
    pool = [(cg.Graph.from_workload_graph(g), eps) for g, eps in wpool]
    build_s = time.perf_counter() - t0
    rng = np.random.default_rng(1234 + rank)
    n_spec = int(args.rate * args.duration * 1.2) + 16
    gids = rng.integers(0, len(pool), n_spec)
    sizes = np.exp(rng.uniform(np.log(1e3), np.log(1e6), n_spec)).astype(np.int64)
    specs = [RequestSpec(int(g), int(sz), 10_000 + q) for q, (g, sz) in enumerate(zip(gids, sizes))]
    budget = int(args.budget_gb * (1 << 30))

    def one(rate, duration):
        res = {}
        forms = [f.strip() for f in args.serving_forms.split(",") if f.strip()]
        rkw = dict(mode=cg.COS_MODE_FP32_MIXED)
        if args.inflight_work is not None:
            rkw["max_inflight_work"] = args.inflight_work
        if args.inflight_max is not None:
            rkw["max_inflight"] = args.inflight_max
        for name, kw in (("resident_mixed", rkw),
                         ("batched_mixed", dict(mode=cg.COS_MODE_FP32_MIXED, max_batch=64, streams=2)),
                         ("plain_fp64", dict(mode=cg.COS_MODE_FP64, single=True))):
            if name.split("_")[0] not in forms:
                continue
            if name.startswith("resident"):
                srv = ResidentScheduler(pool, budget_bytes=budget, max_queue=args.max_queue, **kw)
            else:
                srv = Server(pool, budget_bytes=budget, max_queue=args.max_queue, **kw)
            reqs, wall = poisson_run(srv, specs, rate_per_s=rate, duration_s=duration, seed=rank)
            summ = latency_summary(reqs)
            summ.update({"offered": len(reqs), "shed": int(sum(r.status == "shed" for r in reqs)),
                         "failed": int(sum(r.status == "failed" for r in reqs)), "wall_s": wall,
                         "edge_sample_updates_per_s": srv.units_done / wall,
                         "peak_admitted_gb": (srv.reserved if name.startswith("resident") else srv.ctrl.peak)
                         / (1 << 30)})
            if name.startswith("resident"):
                summ["kernel_launches"] = srv.srv.stats()["launches"]
            if rank == 0 and not args.no_oracle_check:
                summ["error_vs_oracle"] = serving_oracle_check(torch, reqs, wpool, srv.beta, kw["mode"],
                                                               counter=name.startswith("resident"))
            res[name] = summ
            srv.close()
        return res

    out = one(args.rate, args.duration)
    sweep = {}
    for r in [float(x) for x in args.sweep_rates.split(",") if x.strip()]:
        sweep[f"{r:g}_req_per_s"] = one(r, args.sweep_duration)
    for g, _ in pool:
        g.close()
    if rank != 0:
        return None
    b = out.get("resident_mixed") or next(iter(out.values()))
    return {
        "metric": "served edge·sample updates/s", "value": b["edge_sample_updates_per_s"],
        "unit": "edge·sample updates/s", "n_gpus": world, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (sink and sample sums f64)", "data": "synthetic",
        "config": {"workload": f"serving: Poisson {args.rate:g} req/s for {args.duration:g} s; pool of "
                               f"{args.pool_size} leveled DAGs, N logU[1e3,{args.max_nodes:g}], geometric fan-in "
                               f"1..6, K=32, D=L; samples per request logU[1e3,1e6]; budget {args.budget_gb:g} GB; "
                               f"queue bound {args.max_queue}", "pool_build_s": build_s},
        "serving": out, "rate_sweep": sweep,
    }


# ------------------------------------------------------------------ reference arm (the CPU oracle)

def batched_desc(num_graphs: int) -> str:
    return (f"batched uneven: {num_graphs} graphs, order n~U{{2..8}}, L=2n+2, N logU[1e3,1e6], "
            "fan-in U{1..4}, K=16, D=L, samples logU[4096,2^20], one persistent CUDA-graph-captured launch")


def run_reference_batched(args, rank, world):
    """The oracle on the batched workload: each step evaluates the same fraction of
    every graph's samples (its first ones, at least one), so a step has the
    workload's mix of graphs and sample counts; the fraction is sized so that
    warm-up and timed steps take about --reference-seconds (two minutes by default)."""
    if rank != 0:
        return None
    from workloads import batched
    import oracle
    oracle.build()
    wls = batched(seed=3, num_graphs=args.num_graphs)
    t0 = time.perf_counter()
    for w in wls:                                          # rate probe: 4 samples of every graph
        oracle.evaluate(w.graph, w.samples.eps, w.samples.beta, w.samples.t[:4], with_abs=False)
    rate = sum(w.graph.num_edges * min(4, w.samples.num_samples) for w in wls) / (time.perf_counter() - t0)
    total = float(sum(w.graph.num_edges * w.samples.num_samples for w in wls))
    frac = min(1.0, rate * args.reference_seconds / max(1, args.steps + args.warmup) / total)
    n = [max(1, int(frac * w.samples.num_samples)) for w in wls]
    units = float(sum(w.graph.num_edges * k for w, k in zip(wls, n)))

    def step():
        for w, k in zip(wls, n):
            oracle.evaluate(w.graph, w.samples.eps, w.samples.beta, w.samples.t[:k], with_abs=False)

    for _ in range(args.warmup):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    value = units * args.steps / sum(times)
    cores = len(os.sched_getaffinity(0))
    mode_name = args.mode or "mixed"
    return {
        "impl": "reference", "metric": "edge·sample updates/s", "value": value, "unit": "edge·sample updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": batched_desc(len(wls)), "mode": mode_name, "sample_fraction": frac,
                   "edge_samples_per_step": units,
                   "note": "the reference arm is the CPU oracle (plain level-wise DP in double, OpenMP over samples)"},
        "cpu_baseline": {"value": value, "unit": "edge·sample updates/s", "cores": cores, "kind": "oracle",
                         "sample": f"the first {frac:.2e} of every graph's samples per step"},
        "e2e": {"value": value, "unit": "edge·sample updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_reference(args, rank, world):
    if rank != 0:
        return None
    factory, default_mode, desc = WORKLOADS[args.workload]
    mode_name = args.mode or default_mode
    kw = {} if args.samples is None else {"num_samples": args.samples}
    wl = factory(**kw)
    g, s = wl.graph, wl.samples
    import oracle
    oracle.build()
    # size each step so that warmup + steps take about --reference-seconds in total
    n = 8
    t0 = time.perf_counter()
    oracle.evaluate(g, s.eps, s.beta, s.t[:n], with_abs=False)
    per = (time.perf_counter() - t0) / n
    n_step = int(max(8, min(s.num_samples, args.reference_seconds / max(per, 1e-9) / max(1, args.steps + args.warmup))))
    for k in range(args.warmup):
        oracle.evaluate(g, s.eps, s.beta, s.t[:n_step], with_abs=False)
    times = []
    for k in range(args.steps):
        lo = (k * n_step) % max(1, s.num_samples - n_step + 1)
        t0 = time.perf_counter()
        oracle.evaluate(g, s.eps, s.beta, s.t[lo:lo + n_step], with_abs=False)
        times.append(time.perf_counter() - t0)
    value = g.num_edges * n_step * args.steps / sum(times)
    cores = len(os.sched_getaffinity(0))
    return {
        "impl": "reference", "metric": "edge·sample updates/s", "value": value, "unit": "edge·sample updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded random leveled DAG and uniform sample times)",
        "config": {"workload": desc, "mode": mode_name, "samples_per_step": n_step,
                   "note": "the reference arm is the CPU oracle (plain level-wise DP in double, OpenMP over samples)"},
        "cpu_baseline": {"value": value, "unit": "edge·sample updates/s", "cores": cores, "kind": "oracle",
                         "sample": f"{n_step} samples per step of the {args.workload} workload"},
        "e2e": {"value": value, "unit": "edge·sample updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main(argv=None):
    argv = sys.argv[1:] if argv is None else list(argv)
    args = parse_args(argv)
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        return launch_ranks(args.gpus, argv)
    rank, world, local = dist_env()
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if args.impl == "reference":
            # only rank 0 runs the oracle; the other ranks exit at once without work
            if rank != 0:
                return 0
        else:
            dist.init_process_group(backend=backend)
    if args.impl == "reference":
        if args.workload == "serving":
            line = {"impl": "reference", "unavailable": "the serving workload has no CPU reference arm"} if rank == 0 else None
        elif args.workload == "batched":
            line = run_reference_batched(args, rank, world)
        else:
            line = run_reference(args, rank, world)
    elif args.workload == "serving":
        line = run_serving(args, rank, world, local)
    elif args.workload == "batched":
        line = run_batched(args, rank, world, local)
    else:
        line = run_ours(args, rank, world, local)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1 and args.impl != "reference":
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
