"""Benchmark of the fused fluctuating D2Q9 step on GB300.

One benchmark step = one pass of the whole hot path over the 4096x4096 FP32
lattice: pull streaming, density and velocity, the per-node basis, relaxation,
Philox noise, back transform and store (the step kernel), with the equal-time
correlation sums sampled on every step and added to the FP64 accumulators, both
inside the step kernel (one launch per step). Inputs (two 604 MB population
buffers) are larger than L2 and stay resident in HBM.

Prints one JSON line. Multi-GPU runs are independent replicas (one lattice per
rank, weak scaling); ranks only meet at the barriers around the timed region.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS & % of HBM roofline (FP32 vs FP64); batched replica-steps/s, p50/p99"
UNIT = "MLUPS"
BYTES_PER_NODE = {"fp32": 72, "fp64": 144}
# DRAM bytes (read + write) per launch of the FP32 step kernel at 4096^2,
# f-norm basis, sampling every step (tensor-core sums, 12 colliding warps):
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one 2048^2 launch of
# the same kernel (156.3 + 101.4 MB) times the 4x nodes; a full-size capture
# may take only the launch list. Valid only for the kernel version it was
# taken on.
DRAM_TRAFFIC = {("fp32", "local", 4096): 4 * (156.00e6 + 101.18e6),
                ("fp32", "lut", 4096): 4 * (156.00e6 + 102.08e6)}
TRAFFIC_SOURCE = "ncu dram bytes of a 2048^2 launch of the same kernel, x 4 (the nodes)"
# FP64 operations per node-step of the FP64 step kernel (f-norm, sampling
# every step): 2 DFMA + DADD + DMUL thread instructions counted by ncu on a
# 2048^2 launch (388 + 118 + 176 per node; the FP64 pipe 87 % busy). The
# FP64 kernel is bound by GB300's FP64 rate, not by HBM: its roofline is
# reported against the nominal FP64 peak (there is no measured FP64 peak).
FP64_FLOPS_PER_NODE = {"local": 1070.0}
FP64_NOMINAL_TFLOPS = 1.25
# Warp instructions per node-step of the FP32 step kernel with sampling every
# step (tensor-core sums, 16 colliding warps), from ncu smsp__inst_executed.sum
# of a 2048^2 launch (51.9 M and 53.7 M over 4.19 M nodes): with the issue rate
# of the GPU (4 schedulers per SM, one warp instruction per cycle each) they
# give the issue ceiling the f-norm step is bound by.
INSTR_PER_NODE = {("fp32", "local"): 12.37, ("fp32", "lut"): 12.80}
SCHEDULERS_PER_SM = 4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--basis", default="local", choices=["local", "standard", "lut"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--ux0", type=float, default=0.1)
    ap.add_argument("--side", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--pipeline-warps", type=int, default=0,
                    help="consumer warps of the pipelined FP32 kernel (8 or 12; 0 = library default)")
    ap.add_argument("--pipeline-sampling", type=int, default=0,
                    help="1: sampler warps, 2: sums fused into the colliding warps (0 = default)")
    ap.add_argument("--sample-every", type=int, default=1,
                    help="sample the correlations every k steps (1 = every step, the workload)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched-ensemble comparison added to the JSON line")
    ap.add_argument("--batched-steps", type=int, default=200)
    ap.add_argument("--workload", default="single",
                    choices=["single", "ensemble", "serving", "precision", "sweep", "sweep21",
                             "structure"],
                    help="single: the 4096^2 lattice (with the ensemble comparison added); "
                         "ensemble: only the batched replica ensemble, as the main line")
    ap.add_argument("--replicas", type=int, default=256, help="replicas of the ensemble")
    ap.add_argument("--serve-requests", type=int, default=128,
                    help="requests of the serving trace (its first N) served in each mode")
    ap.add_argument("--serve-pool-gb", type=float, default=16.0,
                    help="device pool of the server: the HBM budget admission works against")
    ap.add_argument("--serve-slots", type=int, default=256)
    ap.add_argument("--serve-chunk", type=int, default=16)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-other-basis", action="store_true",
                    help="skip timing the same lattice in the other basis")
    ap.add_argument("--no-per-lattice", action="store_true",
                    help="skip the one-launch-per-lattice arm of the ensemble comparison")
    ap.add_argument("--graph-steps", type=int, default=25)
    ap.add_argument("--no-structure", action="store_true",
                    help="skip the structure-factor sampling measurement")
    ap.add_argument("--structure-steps", type=int, default=100)
    ap.add_argument("--min-seconds", type=float, default=1.0,
                    help="repeat the timed block of --steps steps until it spans this much device time")
    ap.add_argument("--max-repeats", type=int, default=1000)
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 kernel measurement")
    ap.add_argument("--no-precision", action="store_true", help="skip the precision study")
    ap.add_argument("--precision-side", type=int, default=8192)
    ap.add_argument("--no-serving-70", action="store_true",
                    help="skip the serving run at 70 %% of the measured capacity")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def smi_id(dev):
    """nvidia-smi identifier of torch device `dev` (honours CUDA_VISIBLE_DEVICES)."""
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").strip()
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if dev < len(ids):
            return ids[dev]
    return str(dev)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_model():
    """Model name of the host CPU (lscpu; /proc/cpuinfo as a fallback)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for ln in fh:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_runs(p, side, steps, threads, precision="fp64"):
    """The oracle as it stands (plain FP64 C, one lattice per host thread) on
    `threads` independent side x side lattices of the workload's parameters
    with distinct seeds, `steps` steps each with sampling on; ctypes releases
    the GIL, so the threads run on separate cores. Returns aggregate MLUPS and
    the wall time."""
    import concurrent.futures as cf

    import oracle as O
    from paper_1204_6734_gb300 import inputs
    runs = [O.Run(inputs.LatticeParams(side, side, p.rho0, p.ux0, p.uy0, p.kT, p.omega, p.basis,
                                       precision, seed=p.seed + 7919 * k), warmup=0, every=1)
            for k in range(threads)]
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(threads) as ex:
        list(ex.map(lambda r: r.step(steps), runs))
    dt = time.perf_counter() - t0
    return threads * side * side * steps / dt / 1e6, dt


def oracle_mlups(p, max_seconds=15.0, side=1024):
    """The CPU baseline of the line: the oracle on every host core at once, one
    independent side x side lattice per core, with the step count calibrated
    (one step on one core) to about max_seconds of wall time."""
    cores = host_cores()
    one, dt1 = oracle_runs(p, side, 1, 1)
    n = max(1, int(max_seconds / max(dt1, 1e-6)))
    v, dt = oracle_runs(p, side, n, cores)
    sample = (f"{cores} independent {side}x{side} lattices of the workload's parameters (FP64 "
              f"oracle, one per host thread, distinct seeds), {n} steps each with sampling on, "
              f"{dt:.1f} s wall; CPU: {cpu_model()}; one thread alone: {one:.2f} MLUPS")
    return v, sample, cores


def bench_structure(args, p, stream, peak, peak_kind):
    """Cost of one structure-factor sample (Eqs. sfactorr, sfactoru,
    rcorrelator) on the bench lattice: steps with S_k sampled every step minus
    steps without, per step. Algorithmic bytes of the power-of-two FP32 path
    per node: the step kernel writes the sampled state's three fields (12); the
    row kernel reads them (12) and writes the half spectrum (12); the column
    kernel reads it (12) and reads and writes the FP32 partial sums (16); the
    flush of the partials into the FP64 sums every 16 samples (2.5 amortised):
    66.5 B."""
    import torch

    from paper_1204_6734_gb300 import flb

    n = args.structure_steps
    nodes = p.Lx * p.Ly
    with flb.Lattice(p, stream=stream) as lat:
        lat.set_sampling(0, args.sample_every)
        lat.step(5)
        lat.sync()

        def timed():
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.step(n)
            e1.record(stream)
            lat.sync()
            return e0.elapsed_time(e1) / n

        base = timed()
        lat.set_structure_sampling(0, 1)
        lat.step(3)
        lat.sync()
        with_sk = timed()
        ns = lat.structure_factors()[3]
    per = with_sk - base
    pow2 = p.Lx & (p.Lx - 1) == 0 and p.Ly & (p.Ly - 1) == 0 and max(p.Lx, p.Ly) <= 4096
    out = {"ms_per_sample": per, "ms_per_step": base, "ms_per_step_sampled": with_sk,
           "samples": ns, "path": "power-of-two (2 launches)" if pow2 else "general"}
    if pow2 and p.precision == "fp32":
        b = 66.5 * nodes
        ach = b / (per * 1e-3) / 1e9
        out["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                           "frac": ach / peak, "peak_kind": peak_kind, "algorithmic_bytes": b,
                           "bytes_per_node": 66.5,
                           "kernels": "field stores in step_tma_kernel + rows_fields_kernel + "
                                      "cols_part_kernel + flush_part4_kernel"}
    return out


def bench_batched(args, stream):
    """The uneven-replica ensemble (256 lattices, sides log-uniform in
    [64, 1024], FP32, f-norm basis, correlations sampled every step) two ways:
    one persistent launch per step for the whole batch (CUDA graph, tile shape
    chosen by the autotuner), and one launch per lattice per step (a lattice
    handle each). Replica-steps per second of both, on the same stream."""
    import torch

    from paper_1204_6734_gb300 import flb, inputs
    ps = inputs.replica_ensemble(n=args.replicas)
    nodes = sum(p.Lx * p.Ly for p in ps)
    out = {"workload": f"{len(ps)} periodic replicas, sides log-uniform in [64, 1024], u_x0 ~ U[0, 0.3], "
                       "kT in {1e-5, 1e-4, 1e-3}, shear rate ~ U[0.6, 1.8], FP32, local basis, "
                       "sampled every step",
           "replicas": len(ps), "nodes": nodes}

    def timed(fn, k):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            e0.record(stream)
            fn(k)
            e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e-3

    with flb.Batch(ps, stream=stream) as b:
        b.set_sampling(0, 1)
        tile, ms = b.autotune(trial_steps=10)
        b.set_graph(args.graph_steps)
        b.step(args.graph_steps)          # capture + warm
        b.sync()
        k = max(args.graph_steps, args.batched_steps // args.graph_steps * args.graph_steps)
        dt = timed(b.step, k)
        b.sync()
        out.update({"replica_steps_per_s": len(ps) * k / dt, "mlups": nodes * k / dt / 1e6,
                    "steps": k, "ms_per_step": dt / k * 1e3, "graph_steps": args.graph_steps,
                    "tile": [t for t, v in flb.TILE.items() if v == tile][0],
                    "autotune_ms_per_step": dict(zip(flb.TILE, [float(x) for x in ms])),
                    "gpu_launches_per_step": 1})
    peak, kind = measured_peaks()
    achieved = BYTES_PER_NODE["fp32"] * nodes / (dt / k) / 1e9
    out["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                       "frac": achieved / peak, "peak_kind": kind,
                       "kernel": "batch_step_kernel<local,sample>"}

    if args.no_per_lattice:
        return out
    # the same replicas as lattice handles, one launch per lattice and step:
    # driven from Python (what a caller of the one-lattice API does), and
    # captured into one CUDA graph (no host overhead left: the GPU cost of
    # one launch per lattice)
    lats = [flb.Lattice(p, stream=stream, kernel="pipelined") for p in ps]
    try:
        for lat in lats:
            lat.set_sampling(0, 1)

        def per_lattice(k):
            for _ in range(k):
                for lat in lats:
                    flb.flb_step(lat.h, 1)
        per_lattice(2)
        k1 = max(5, args.batched_steps // 10)
        dt1 = timed(per_lattice, k1)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            per_lattice(k1)
        with torch.cuda.stream(stream):
            g.replay()
        dt2 = timed(lambda k: g.replay(), k1)
        for lat in lats:
            lat.sync()
        del g
    finally:
        for lat in lats:
            lat.close()
    out["one_lattice_per_launch"] = {"replica_steps_per_s": len(ps) * k1 / dt1,
                                     "mlups": nodes * k1 / dt1 / 1e6, "steps": k1,
                                     "ms_per_step": dt1 / k1 * 1e3, "gpu_launches_per_step": len(ps),
                                     "driver": "python loop of flb_step"}
    out["one_lattice_per_launch_graph"] = {"replica_steps_per_s": len(ps) * k1 / dt2,
                                           "mlups": nodes * k1 / dt2 / 1e6, "steps": k1,
                                           "ms_per_step": dt2 / k1 * 1e3,
                                           "gpu_launches_per_step": len(ps),
                                           "driver": "the same launches captured in one CUDA graph"}
    out["speedup"] = out["replica_steps_per_s"] / out["one_lattice_per_launch"]["replica_steps_per_s"]
    out["speedup_vs_graph"] = out["replica_steps_per_s"] / \
        out["one_lattice_per_launch_graph"]["replica_steps_per_s"]
    return out


def serve_trace(args, stream, mode, reqs):
    """Serve a trace of requests (Poisson arrivals replayed in real time: each
    is submitted once its arrival time has passed on the server clock) until
    all have finished. Latency = completion seen by the host - arrival."""
    from paper_1204_6734_gb300 import flb
    pool = int(args.serve_pool_gb * (1 << 30))
    with flb.Server("local", pool, args.serve_slots, args.serve_chunk, mode=mode,
                    stream=stream) as s:
        t_start = s.stats()["clock_s"]
        t_first = reqs[0].arrival_s
        arrival, results, i, n = {}, [], 0, len(reqs)
        while len(results) < n:
            now = s.stats()["clock_s"] - t_start
            while i < n and reqs[i].arrival_s - t_first <= now:
                q = reqs[i]
                rid = s.submit(q.params, q.steps, q.warmup, q.every)
                arrival[rid] = t_start + q.arrival_s - t_first
                i += 1
            got = s.poll(wait=(i == n))
            results += got
            if not got and i < n:
                time.sleep(0.0005)
        st = s.stats()
    lat = sorted(r["t_done"] - arrival[r["id"]] for r in results)
    wall = max(r["t_done"] for r in results) - t_start

    def pct(q):
        return lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)]
    return {"mode": mode, "requests": n, "wall_s": wall,
            "replica_steps_per_s": st["replica_steps"] / wall,
            "mlups": st["node_steps"] / wall / 1e6,
            "latency_p50_s": pct(0.50), "latency_p99_s": pct(0.99), "latency_mean_s": sum(lat) / n,
            "gpu_busy_s": st["gpu_busy_s"], "chunks": st["chunks"],
            "failed": sum(1 for r in results if r["status"] != 0)}


def bench_serving(args, stream, modes=("batched", "per_lattice"), rate_hz=200.0):
    from paper_1204_6734_gb300 import inputs
    reqs = inputs.serving_requests(n=args.serve_requests, rate_hz=rate_hz)
    out = {"workload": f"first {len(reqs)} requests of the serving trace: Poisson arrivals at {rate_hz:.3g}/s, "
                       "sides log-uniform in [32, 2048], u_x0 ~ U[0, 0.3], kT log-uniform in "
                       "[1e-5, 1e-3], shear rate ~ U[0.6, 1.8], steps in [500, 20000], FP32, "
                       "local basis, sampled every step after a tenth of the steps",
           "pool_gb": args.serve_pool_gb, "slots": args.serve_slots, "chunk_steps": args.serve_chunk,
           "node_steps": sum(r.steps * r.params.Lx * r.params.Ly for r in reqs)}
    for m in modes:
        out[m] = serve_trace(args, stream, m, reqs)
    if "batched" in out and "per_lattice" in out:
        out["speedup"] = out["batched"]["replica_steps_per_s"] / out["per_lattice"]["replica_steps_per_s"]
    return out


def run_ensemble(args, rank, world, dist, dev):
    """--workload ensemble: the batched replica ensemble as the main line
    (replica-steps/s; --steps batch steps timed after --warmup)."""
    import torch
    stream = torch.cuda.Stream(device=dev)
    args.batched_steps = args.steps
    with ClockSampler(smi_id(dev)) as clk:
        b = bench_batched(args, stream)
    if rank == 0:
        out = {"metric": METRIC, "value": b["replica_steps_per_s"], "unit": "replica-steps/s",
               "n_gpus": world, "steps": b["steps"], "warmup": args.warmup,
               "ms_per_step": b["ms_per_step"], "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "f32", "data": "synthetic",
               "config": {"workload": b["workload"], "replicas": b["replicas"], "nodes": b["nodes"],
                          "l2": "inputs larger than L2"},
               "roofline": b["roofline"], "batched": b, "clocks": clk.summary(),
               "gpu_launches": b["steps"]}
        print(json.dumps(out))


def run_serving(args, rank, world, dist, dev):
    """--workload serving: the request trace through the server as the main
    line (replica-steps/s with p50/p99 latency)."""
    import torch
    stream = torch.cuda.Stream(device=dev)
    modes = ("batched",) if args.no_per_lattice else ("batched", "per_lattice")
    with ClockSampler(smi_id(dev)) as clk:
        sv = bench_serving(args, stream, modes)
        # the same requests arriving at 70 % of the batched server's measured
        # node-update capacity (the overload run above)
        work = sv["node_steps"] / args.serve_requests
        rate70 = 0.7 * sv["batched"]["mlups"] * 1e6 / work
        sv["at_70pct_capacity"] = bench_serving(args, stream, modes, rate_hz=rate70)
    if rank == 0:
        b = sv["batched"]
        out = {"metric": METRIC, "value": b["replica_steps_per_s"], "unit": "replica-steps/s",
               "n_gpus": world, "steps": None, "warmup": 0, "ms_per_step": None,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic", "config": {"workload": sv["workload"], "l2": "inputs larger than L2"},
               "latency_p50_s": b["latency_p50_s"], "latency_p99_s": b["latency_p99_s"],
               "serving": sv, "clocks": clk.summary()}
        print(json.dumps(out))


def bench_precision(stream, side, steps):
    """The same lattice (u_x0 = 0.2, kT = 1e-4, all rates 1, f-norm, seed 4) run
    `steps` steps in FP64, FP32 and the FP16 deviation store with the same
    draws, sampled every step after a tenth of the steps; errors of the FP32 and
    FP16 states and of <df_i df_j>, <dM dM> against the FP64 run, and the
    throughput of each (CUDA events on the launching stream)."""
    import numpy as np
    import torch

    from paper_1204_6734_gb300 import flb, inputs
    warm = steps // 10
    lats, res = {}, {}
    try:
        for prec in ("fp64", "fp32", "fp16dev"):
            p = inputs.precision_lattice(prec, side=side)
            lat = flb.Lattice(p, stream=stream)
            lats[prec] = lat
            lat.set_sampling(warm, 1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            lat.step(steps)
            e1.record(stream)
            lat.sync()
            ms = e0.elapsed_time(e1) / steps
            Cff, CMM, mean, n = lat.correlations("local")
            res[prec] = {"ms_per_step": ms, "mlups": p.Lx * p.Ly / ms / 1e3,
                         "bytes_per_node": {"fp64": 144, "fp32": 72, "fp16dev": 36}[prec],
                         "Cff": Cff, "CMM": CMM, "n_samples": n}
        kT, wmax = 1e-4, 4.0 / 9.0
        out = {"workload": f"{side}x{side} periodic, u_x0=0.2, kT=1e-4, all rates 1, f-norm basis, "
                           f"seed 4, {steps} steps, sampled every step after {warm}; errors against "
                           "the FP64 run on the GPU (same draws)",
               "steps": steps, "n_samples": int(res["fp32"]["n_samples"])}
        for prec in ("fp64", "fp32", "fp16dev"):
            r = res[prec]
            o = {"mlups": r["mlups"], "ms_per_step": r["ms_per_step"],
                 "bytes_per_node": r["bytes_per_node"]}
            if prec != "fp64":
                mx, rms, fmax = flb.flb_state_difference(lats[prec].h, lats["fp64"].h)
                o["population_error_max"] = mx
                o["population_error_rms"] = rms
                o["corr_error_max_over_kT_wmax"] = float(
                    np.abs(r["Cff"] - res["fp64"]["Cff"]).max() / (kT * wmax))
                o["moment_corr_error_max_over_kT"] = float(
                    np.abs(r["CMM"] - res["fp64"]["CMM"]).max() / kT)
            out[prec] = o
    finally:
        for lat in lats.values():
            lat.close()
    return out


def run_precision(args, rank, world, dist, dev):
    """--workload precision: bench_precision on the 8192^2 lattice (--side) for
    --steps steps, as the main line."""
    import torch
    stream = torch.cuda.Stream(device=dev)
    side = args.side if args.side != 4096 else 8192
    with ClockSampler(smi_id(dev)) as clk:
        out = bench_precision(stream, side, args.steps)
    if rank == 0:
        line = {"metric": METRIC, "value": out["fp32"]["mlups"], "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": 0, "ms_per_step": out["fp32"]["ms_per_step"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": "precision study: " + out["workload"],
                           "l2": "inputs larger than L2"},
                "precision": out, "clocks": clk.summary(), "n_samples": out["n_samples"]}
        print(json.dumps(line))


def bench_fp64(stream, p64, steps, peak, peak_kind):
    """The FP64 parity-mode kernel on the bench lattice (f-norm or Hermite,
    sampling every step): MLUPS, against the FP64 pipe (its bound) and HBM."""
    import torch

    from paper_1204_6734_gb300 import flb
    nodes = p64.Lx * p64.Ly
    with flb.Lattice(p64, stream=stream) as lat:
        lat.set_sampling(0, 1)
        lat.step(2)
        lat.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        lat.sync()
        ms = e0.elapsed_time(e1) / steps
    hbm = BYTES_PER_NODE["fp64"] * nodes / (ms * 1e-3) / 1e9
    out = {"workload": f"{p64.Lx}x{p64.Ly}, FP64 populations, the same parameters, sampled every step",
           "mlups": nodes / ms / 1e3, "ms_per_step": ms, "steps": steps,
           "kernel": "step_kernel<f64,%s,sample>" % p64.basis,
           "hbm": {"achieved": hbm, "peak": peak, "unit": "GB/s", "frac": hbm / peak,
                   "peak_kind": peak_kind}}
    fl = FP64_FLOPS_PER_NODE.get(p64.basis)
    if fl:
        tf = fl * nodes / (ms * 1e-3) / 1e12
        out["roofline"] = {"bound": "alu", "achieved": tf, "peak": FP64_NOMINAL_TFLOPS,
                           "unit": "TFLOP/s", "frac": tf / FP64_NOMINAL_TFLOPS,
                           "peak_kind": "nominal FP64 rate (no measured FP64 peak)",
                           "flops_per_node": fl}
    return out


MOMENT_NAMES = ("rho", "j_x", "j_y", "Pi_xx-yy", "Pi_xy", "Pi_xx+yy", "q_x", "q_y", "eps")   # drift.MOMENTS
# Quadratic coefficients q the paper prints for 21x21 lattices (Section 4,
# after Figs. 19-21): Hermite norm measured in the Hermite norm, f-norm (its
# look-up-table variant) measured in the f-norm at u0.
PAPER_Q = {"standard": {"rho": 1.9, "Pi_xx-yy": 1.6, "j_y": 1.14},
           "local": {"rho": 0.47, "Pi_xx-yy": 0.54, "j_y": 0.75},
           "lut": {"rho": 0.47, "Pi_xx-yy": 0.54, "j_y": 0.75}}


def run_sweep(args, rank, world, dist, dev):
    """--workload sweep: the u_x0 sweep of the 4096^2 lattice in both bases
    (--steps steps each, sampled every step after a tenth); the normalised
    moment correlators <dM^a dM^b> / (kT rho0) - delta^{ab}, measured in the
    run's own basis at u0, and the paper's fit l u + q u^2 of all 45 of them
    (paper_1204_6734_gb300.drift)."""
    import numpy as np
    import torch

    from paper_1204_6734_gb300 import drift, flb, inputs
    stream = torch.cuda.Stream(device=dev)
    warm = max(1, args.steps // 10)
    res = {}
    with ClockSampler(smi_id(dev)) as clk:
        for basis in ("standard", "local", "lut"):
            rows = []
            mb = "standard" if basis == "standard" else "local"
            for u in inputs.SWEEP_UX0:
                p = inputs.single_lattice(u, basis, side=args.side)
                with flb.Lattice(p, stream=stream) as lat:
                    lat.set_sampling(warm, 1)
                    lat.step(args.steps)
                    lat.sync()
                    Cff, CMM, mean, n = lat.correlations(mb)
                rows.append((u, drift.normalised(CMM, p.kT, p.rho0),
                             np.diag(Cff) / (p.kT * feq_of(p))))
            us = np.array([r[0] for r in rows])
            DM = np.array([r[1] for r in rows])
            D = np.array([np.diag(m) for m in DM])
            l, q = drift.fit_lq(us, DM)
            res[basis] = {
                "u_x0": [float(u) for u in us],
                "moment_variance_minus_1": {MOMENT_NAMES[a]: [float(x) for x in D[:, a]] for a in range(9)},
                "population_variance_over_kT_f0": [[float(x) for x in r[2]] for r in rows],
                "fit_q": {MOMENT_NAMES[a]: float(q[a, a]) for a in range(9)},
                "fit_lq": drift.as_table(l, q),
                "max_abs_l_odd_pairs": float(np.abs(l).max()),
                "paper_q_21x21": PAPER_Q[basis],
            }
    if rank == 0:
        line = {"metric": METRIC, "value": None, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": warm, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"u_x0 sweep {list(inputs.SWEEP_UX0)} of the {args.side}^2 "
                                       "lattice (kT=1e-4, shear 1.0, bulk 0.8, ghost 1.0), both bases, "
                                       f"sampled every step after {warm}",
                           "l2": "inputs larger than L2"},
                "sweep": res, "clocks": clk.summary()}
        print(json.dumps(line))


def run_sweep21(args, rank, world, dist, dev):
    """--workload sweep21: the u_x0 sweep on the paper's own 21 x 21 lattice.
    --replicas independent copies per (u_x0, basis), all points of one basis in
    one batch (one launch per step), --steps steps sampled every step after a
    tenth; the moment variances of the pooled copies (flb_batch_correlations)
    fitted as in the 4096^2 sweep, in the Hermite norm, the local f-norm and
    the table f-norm (the variant the paper's f-norm numbers come from)."""
    import numpy as np
    import torch

    from paper_1204_6734_gb300 import drift, flb, inputs
    stream = torch.cuda.Stream(device=dev)
    warm = max(1, args.steps // 10)
    R = args.replicas
    res = {}
    with ClockSampler(smi_id(dev)) as clk:
        for basis in ("standard", "local", "lut"):
            ps = [p for u in inputs.SWEEP_UX0 for p in inputs.small_sweep_replicas(u, basis, R)]
            with flb.Batch(ps, stream=stream) as b:
                b.set_sampling(warm, 1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                b.step(args.steps)
                e1.record(stream)
                b.sync()
                ms = e0.elapsed_time(e1)
                rows = []
                for iu, u in enumerate(inputs.SWEEP_UX0):
                    slots = list(range(iu * R, (iu + 1) * R))
                    Cff, CMM, mean, n = b.correlations(slots, "standard" if basis == "standard" else "local")
                    p = ps[iu * R]
                    rows.append((u, drift.normalised(CMM, p.kT, p.rho0), n))
            us = [r[0] for r in rows]
            DM = np.array([r[1] for r in rows])
            D = np.array([np.diag(m) for m in DM])
            l, q = drift.fit_lq(us, DM)
            nodes = sum(p.Lx * p.Ly for p in ps)
            res[basis] = {
                "u_x0": us, "node_samples_per_point": [int(r[2]) for r in rows],
                "moment_variance_minus_1": {MOMENT_NAMES[a]: [float(x) for x in D[:, a]] for a in range(9)},
                "fit_q": {MOMENT_NAMES[a]: float(q[a, a]) for a in range(9)},
                "fit_lq": drift.as_table(l, q),
                "max_abs_l_odd_pairs": float(np.abs(l).max()),
                "paper_q_21x21": PAPER_Q[basis],
                "batch_ms_per_step": ms / args.steps, "mlups": nodes * args.steps / (ms * 1e-3) / 1e6,
            }
    if rank == 0:
        line = {"metric": METRIC, "value": None, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": warm, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"u_x0 sweep {list(inputs.SWEEP_UX0)} on 21x21 lattices, {R} "
                                       "independent copies per point pooled (kT=1e-4, shear 1.0, bulk 0.8, "
                                       f"ghost 1.0), Hermite, f-norm and table f-norm, sampled every step "
                                       f"after {warm}",
                           "l2": "state fits L2 (small lattices)"},
                "sweep21": res, "clocks": clk.summary()}
        print(json.dumps(line))


def run_structure(args, rank, world, dist, dev):
    """--workload structure: the anisotropy of the static structure factors
    (Eqs. sfactorr, sfactoru, rcorrelator) at u_x0 = 0, 0.1, 0.2 in both norms
    on a --side^2 lattice (default 64): S_k / (N kT) - 1 for rho and
    S_k / (N kT / 3) - 1 for j_x (0 for the ideal gas at every k != 0), averaged
    over the modes on the k_x axis (m_y = 0), on the k_y axis (m_x = 0) and
    over all k != 0; |R_k| / (N kT / 3) likewise. Thermalised for --warmup
    steps, then --steps steps with S_k sampled every 5."""
    import numpy as np
    import torch

    from paper_1204_6734_gb300 import flb, inputs
    side = args.side if args.side != 4096 else 64
    every = 5
    res = {}
    t0 = time.perf_counter()
    for basis in ("standard", "local"):
        rows = {}
        for u in (0.0, 0.1, 0.2):
            p = inputs.single_lattice(u, basis, side=side)
            with flb.Lattice(p) as lat:
                lat.set_structure_sampling(args.warmup, every)
                lat.step(args.warmup + args.steps)
                Sr, Sx, R, n = lat.structure_factors()
            N = side * side
            a, b, c = Sr / (N * p.kT) - 1.0, Sx / (N * p.kT / 3.0) - 1.0, np.abs(R) / (N * p.kT / 3.0)
            mask = np.ones_like(a, dtype=bool)
            mask[0, 0] = False

            def dirs(x):
                return {"k_x_axis": float(x[0, 1:].mean()), "k_y_axis": float(x[1:, 0].mean()),
                        "all_k": float(x[mask].mean()),
                        "k_x_axis_min": float(x[0, 1:].min()), "k_x_axis_max": float(x[0, 1:].max())}
            rows[str(u)] = {"samples": int(n), "S_rho_minus_1": dirs(a), "S_jx_minus_1": dirs(b),
                            "abs_R": dirs(c)}
        res[basis] = rows
    if rank == 0:
        line = {"metric": METRIC, "value": None, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"structure factors of the {side}^2 lattice (kT=1e-4, shear 1.0, "
                                       "bulk 0.8, ghost 1.0) at u_x0 = 0, 0.1, 0.2, Hermite and f-norm, "
                                       f"sampled every {every} steps after {args.warmup}",
                           "l2": "state fits L2 (small lattice)"},
                "structure": res, "wall_s": time.perf_counter() - t0}
        print(json.dumps(line))


def feq_of(p):
    """f_i^0(rho0, u0) of Eq. d2q9f0, to normalise the measured variances."""
    import numpy as np
    usq = p.ux0 ** 2 + p.uy0 ** 2
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
    cy = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    uv = p.ux0 * cx + p.uy0 * cy
    return p.rho0 * w * (1 + 3 * uv + 4.5 * uv ** 2 - 1.5 * usq)


def single_config(p, args, world):
    """The config object of the single-lattice line (both arms)."""
    return {"workload": f"{p.Lx}x{p.Ly} periodic D2Q9 lattice, {args.precision} SoA, "
                        f"{args.basis} basis, u_x0={p.ux0}, kT={p.kT}, "
                        f"omega shear/bulk/ghost=1.0/0.8/1.0, correlations sampled every step",
            "Lx": p.Lx, "Ly": p.Ly, "basis": args.basis, "precision": args.precision,
            "parallelism": f"replicas x{world}",
            "l2": "inputs larger than L2 (2 x 604 MB population buffers)"}


def run_reference(args):
    """The reference arm: the oracle (the method written plainly from the paper,
    FP64, one lattice per host thread) on every host core, each timed step one
    step of 256x256 lattices of the workload's parameters on every core."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1204_6734_gb300 import inputs
    p = inputs.single_lattice(args.ux0, args.basis, side=args.side, precision="fp64")
    side = 256
    cores = host_cores()
    oracle_runs(p, side, args.warmup, cores)
    value, dt = oracle_runs(p, side, args.steps, cores)
    cfg = single_config(inputs.single_lattice(args.ux0, args.basis, side=args.side,
                                              precision=args.precision), args, world)
    cfg.update({"Lx": side, "Ly": side, "precision": "fp64", "replicas": cores,
                "sample_of": cfg["workload"],
                "workload": f"{cores} independent {side}x{side} periodic D2Q9 lattices (one per "
                            f"host core), FP64 oracle, {args.basis} basis, u_x0={p.ux0}, kT={p.kT}, "
                            "omega shear/bulk/ghost=1.0/0.8/1.0, correlations sampled every step",
                "parallelism": f"host threads x{cores}",
                "l2": "CPU run"})
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / max(args.steps, 1) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": cfg,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{cores} independent {side}x{side} lattices, FP64, one per "
                                   f"host thread, {args.steps} steps each (aggregate MLUPS); "
                                   f"CPU: {cpu_model()}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch

    from paper_1204_6734_gb300 import flb, inputs, replicas

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    flb.load()

    if args.workload != "single" and rank != 0:
        # the ensemble, serving and precision workloads run on one GPU (rank 0)
        dist.barrier()
        dist.destroy_process_group()
        return
    if args.workload != "single":
        if dist is not None:
            dist.barrier()
        run = {"ensemble": run_ensemble, "serving": run_serving, "precision": run_precision,
               "sweep": run_sweep, "sweep21": run_sweep21, "structure": run_structure}
        run[args.workload](args, rank, world, dist, dev)
        if dist is not None:
            dist.destroy_process_group()
        return

    p = replicas.rank_params(
        inputs.single_lattice(args.ux0, args.basis, side=args.side, precision=args.precision), rank)
    nodes = p.Lx * p.Ly
    stream = torch.cuda.Stream(device=dev)
    lat = flb.Lattice(p, stream=stream,
                      pipeline_warps=args.pipeline_warps if args.pipeline_warps else None,
                      pipeline_sampling=args.pipeline_sampling if args.pipeline_sampling else None)
    lat.set_sampling(0, args.sample_every)   # sample (and reduce) every step by default

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up (also gives the length of one step, to size the repeats)
    w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0.record(stream)
    lat.step(args.warmup)
    w1.record(stream)
    lat.sync()
    warm_ms = w0.elapsed_time(w1) / max(args.warmup, 1)
    # the timed region: blocks of exactly --steps steps, each bracketed by a
    # barrier and a device synchronisation, repeated until they span at least
    # --min-seconds of device time (and at least 3 times); the line reports the
    # median block (max over ranks), and the clocks sampled across all of them
    repeats = max(3, int(math.ceil(args.min_seconds * 1e3 / max(warm_ms * args.steps, 1e-3))))
    repeats = min(repeats, args.max_repeats)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all1 = torch.cuda.Event(enable_timing=True)
    block_ms, per_step = [], []
    with ClockSampler(smi_id(dev)) as clk:
        for _ in range(repeats):
            barrier()
            t_all0.record(stream)
            for k in range(args.steps):
                starts[k].record(stream)
                flb.flb_step(lat.h, 1)
                ends[k].record(stream)
            t_all1.record(stream)
            barrier()
            block_ms.append(replicas.max_over_ranks(t_all0.elapsed_time(t_all1), dist, device="cuda"))
            per_step += [a.elapsed_time(b) for a, b in zip(starts, ends)]
    lat.sync()
    total_ms = statistics.median(block_ms)
    value = replicas.whole_job_rate(nodes * args.steps, world, total_ms * 1e-3) / 1e6
    step_ms = statistics.mean(per_step)

    peak, peak_kind = measured_peaks()
    algo_bytes = BYTES_PER_NODE[args.precision] * nodes
    achieved = algo_bytes / (step_ms * 1e-3) / 1e9
    pipelined = args.precision == "fp32"
    kname = ("step_tma_kernel<%s,sample>" % args.basis) if pipelined else \
        ("step_kernel<f64,%s,sample>" % args.basis)
    traffic = DRAM_TRAFFIC.get((args.precision, args.basis, args.side))
    if args.pipeline_warps or args.pipeline_sampling or args.sample_every != 1:
        traffic = None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                "kernel": kname, "algorithmic_bytes": algo_bytes,
                "traffic_source": TRAFFIC_SOURCE if traffic else None}
    ipn = INSTR_PER_NODE.get((args.precision, args.basis))
    if ipn and args.sample_every == 1 and not args.pipeline_warps and not args.pipeline_sampling:
        props = torch.cuda.get_device_properties(dev)
        mhz = clk.summary().get("sm_mhz") or 2070.0
        peak_inst = props.multi_processor_count * SCHEDULERS_PER_SM * mhz * 1e6
        got = ipn * nodes / (step_ms * 1e-3)
        roofline["issue"] = {"instructions_per_node": ipn, "achieved": got / 1e9, "peak": peak_inst / 1e9,
                             "unit": "G warp-instructions/s", "frac": got / peak_inst,
                             "source": "ncu smsp__inst_executed.sum of a 2048^2 launch"}
    if args.precision == "fp64" and args.basis in FP64_FLOPS_PER_NODE:
        tf = FP64_FLOPS_PER_NODE[args.basis] * nodes / (step_ms * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": tf, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                    "frac": tf / FP64_NOMINAL_TFLOPS, "traffic": None,
                    "peak_kind": "nominal FP64 rate (no measured FP64 peak)", "kernel": kname,
                    "flops_per_node": FP64_FLOPS_PER_NODE[args.basis],
                    "hbm": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                            "peak_kind": peak_kind}}

    Cff, CMM, mean, ns = lat.correlations("standard" if args.basis == "standard" else "local")
    lat.close()

    # end to end through the host-buffer entry point: upload the initial state
    # from pinned host memory, run the same number of steps with sampling,
    # copy back the final state and the sums
    e2e = None
    if not args.no_e2e:
        f_host = torch.empty((9, p.Ly, p.Lx), dtype=torch.float64, pin_memory=True)
        f_out = torch.empty((9, p.Ly, p.Lx), dtype=torch.float64, pin_memory=True)
        with flb.Lattice(p) as tmp:        # equilibrium initial state, not timed
            flb.flb_get_populations(tmp.h, p.Lx, p.Ly, out=f_host.numpy())
        barrier()
        t0 = time.perf_counter()
        flb.flb_run_host(p, f_host.numpy(), args.steps, warmup=0, every=1, f_out=f_out.numpy())
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        state_bytes = 9 * nodes * 8
        e2e = {"value": nodes * args.steps / dt / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": state_bytes / args.steps,
               "d2h_bytes_per_step": (state_bytes + 8 * 90) / args.steps,
               "what": "flb_run_host: pinned host state in, steps with sampling, state + sums out"}

    # the same lattice in the other basis (same size, precision and sampling)
    other = None
    if rank == 0 and world == 1 and not args.no_other_basis:
        ob = "standard" if args.basis != "standard" else "local"
        q = replicas.rank_params(inputs.single_lattice(args.ux0, ob, side=args.side,
                                                       precision=args.precision), rank)
        with flb.Lattice(q, stream=stream) as lo:
            lo.set_sampling(0, args.sample_every)
            lo.step(args.warmup)
            lo.sync()
            n_other = min(args.steps, 500)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lo.step(n_other)
            e1.record(stream)
            lo.sync()
            ms_o = e0.elapsed_time(e1) / n_other
        mlups_o = q.Lx * q.Ly / ms_o / 1e3
        ach = BYTES_PER_NODE[args.precision] * q.Lx * q.Ly / (ms_o * 1e-3) / 1e9
        other = {"basis": ob, "mlups": mlups_o, "ms_per_step": ms_o, "steps": n_other,
                 "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                              "frac": ach / peak, "peak_kind": peak_kind}}

    structure = None
    if rank == 0 and world == 1 and not args.no_structure:
        structure = bench_structure(args, p, stream, peak, peak_kind)

    batched = serving = fp64 = precision = None
    if rank == 0 and world == 1 and not args.no_batched and args.precision == "fp32":
        batched = bench_batched(args, stream)
    if rank == 0 and world == 1 and not args.no_serving and args.precision == "fp32":
        serving = bench_serving(args, stream)
        if not args.no_serving_70:
            # the same requests arriving at 70 % of the batched server's
            # measured node-update capacity
            work = serving["node_steps"] / args.serve_requests
            rate70 = 0.7 * serving["batched"]["mlups"] * 1e6 / work
            serving["at_70pct_capacity"] = bench_serving(args, stream, rate_hz=rate70)
    if rank == 0 and world == 1 and not args.no_fp64 and args.precision == "fp32":
        p64 = replicas.rank_params(inputs.single_lattice(args.ux0, args.basis, side=args.side,
                                                         precision="fp64"), rank)
        fp64 = bench_fp64(stream, p64, max(3, min(args.steps, 20)), peak, peak_kind)
    if rank == 0 and world == 1 and not args.no_precision and args.precision == "fp32":
        precision = bench_precision(stream, args.precision_side, max(10, args.steps))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, sample, cores = oracle_mlups(p)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
            "config": single_config(p, args, world),
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": (1 if pipelined else 2) * args.steps * repeats,
            "repeats": repeats,
            "block_ms": block_ms,
            "clocks": clk.summary(),
            "mlups_roofline_frac": value / (peak * 1e9 / BYTES_PER_NODE[args.precision] / 1e6) / world,
            "n_samples": ns,
            "other_basis": other,
            "structure_factors": structure,
            "batched": batched,
            "serving": serving,
            "fp64": fp64,
            "precision": precision,
        }
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
