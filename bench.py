#!/usr/bin/env python
"""Benchmark: subject fibers labelled per second at 4,145,000 fibers x 10,000 centroids.

One step labels the whole synthetic subject (4,145,000 fibers of 21 points, the paper's headline
subject size) against a 500-bundle x 20-centroid atlas through the C ABI, with inputs resident
in HBM (1.04 GB of fibers, larger than L2). Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--mode plain|gemm_bf16|gemm_tf32]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Multi-GPU: one process per GPU (torchrun); every rank labels its own full subject (weak
scaling, no data-path collective); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "subject fibers labelled/sec at 4.1M fibers (plain vs GEMM-pruned), % of roofline"
UNIT = "fibers/s"
WORKLOAD = "subject4145k_atlas10k"
PAPER_CONTEXT = "paper: 4,145,000 fibers in about 6 min on an i7-6700K (about 11,500 fibers/s)"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--mode", default="plain", choices=["plain", "gemm_bf16", "gemm_tf32"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--config", type=int, default=None, help="tile-shape config (default: tuned)")
    p.add_argument("--n", type=int, default=None, help="override the fiber count")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    return p.parse_args()


# ----------------------------------------------------------------------------- clocks
class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = []
        mx = 0.0
        reasons = set()
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle
def oracle_sample_rate(atlas, fib, seconds: float, seed: int = 0):
    """Time the oracle's paper-order cascade on a random sample sized for about `seconds` of
    CPU work; returns (fibers/s, sample size, threads, point distances per pair)."""
    import oracle
    rng = np.random.default_rng(seed)
    n0 = min(len(fib), 2000)
    idx = rng.choice(len(fib), size=n0, replace=False)
    t = time.perf_counter()
    r = oracle.label(fib[idx], atlas.centroids, atlas.bundle_of, atlas.thresholds, "cascade")
    dt = time.perf_counter() - t
    n1 = int(min(len(fib), max(n0, n0 * seconds / max(dt, 1e-3))))
    idx = rng.choice(len(fib), size=n1, replace=False)
    t = time.perf_counter()
    r = oracle.label(fib[idx], atlas.centroids, atlas.bundle_of, atlas.thresholds, "cascade")
    dt = time.perf_counter() - t
    c = r["counts"]
    return n1 / dt, n1, oracle.max_threads(), float(c[:4].sum()) / float(c[4]), dt


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def traffic_for(kernel: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if it matches."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            t = json.load(fh)
        return t.get(kernel)
    except (OSError, ValueError):
        return None


# ----------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from paper_1912_11494_gb300 import synth
    atlas, fib = synth.workload(args.workload, n=args.n, device="cpu") if args.n and \
        args.n <= 200_000 else _ref_inputs(args)
    per_step = max(1.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    import oracle
    rng = np.random.default_rng(0)
    # size the per-step sample once
    rate, n1, cores, pdpp, _ = oracle_sample_rate(atlas, fib, per_step)
    times = []
    for s in range(args.warmup + args.steps):
        idx = rng.choice(len(fib), size=n1, replace=False)
        t = time.perf_counter()
        oracle.label(fib[idx], atlas.centroids, atlas.bundle_of, atlas.thresholds, "cascade")
        dt = time.perf_counter() - t
        if s >= args.warmup:
            times.append(dt)
    ms = 1000.0 * statistics.mean(times)
    value = n1 / (ms / 1000.0)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "fibers": 4_145_000 if args.n is None else args.n,
                       "centroids": atlas.M, "bundles": atlas.B, "points": 21,
                       "sample_fibers_per_step": n1},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{n1} random fibers of the workload per step against "
                                       f"all {atlas.M} centroids, FP64 progressive-discarding "
                                       f"cascade (Section 2.3)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "context": PAPER_CONTEXT}
    print(json.dumps(line), flush=True)
    return 0


def _ref_inputs(args):
    from paper_1912_11494_gb300 import synth
    # the oracle only needs a sample, so draw the same workload on whatever device exists
    dev = "cuda" if _has_cuda() else "cpu"
    return synth.workload(args.workload, n=args.n, device=dev)


def _has_cuda():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


# ----------------------------------------------------------------------------- our arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    from paper_1912_11494_gb300 import binding, build, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    build.build()

    atlas_np, fib_np = synth.workload(args.workload, n=args.n, device=dev)
    n = int(fib_np.shape[0])
    at = binding.Atlas(torch.as_tensor(atlas_np.centroids, device=dev),
                       torch.as_tensor(atlas_np.bundle_of, device=dev),
                       torch.as_tensor(atlas_np.thresholds, device=dev))
    if args.config is not None:
        binding.seg_set_config(at, args.mode, args.config)
    fib = torch.as_tensor(fib_np, device=dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    dst = torch.empty(n, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        binding.seg_label(at, fib, args.mode, labels, dst, stream=stream)

    for _ in range(max(3, args.warmup)):
        step()
    binding.seg_sync_status(at, stream)
    launches_per_step = 1 if args.mode == "plain" else None

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    clocks = Clocks(local)
    barrier()
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    binding.seg_sync_status(at, stream)
    ms = e0.elapsed_time(e1) / args.steps
    t = torch.tensor([ms], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * n / (ms_max / 1000.0)

    stats = binding.seg_gemm_stats(at) if args.mode != "plain" else None

    # end to end through the public API: pinned host fibers in, labels + distances out
    e2e = None
    if not args.no_e2e:
        h_fib = torch.empty_like(fib, device="cpu").pin_memory()
        h_fib.copy_(torch.as_tensor(fib_np))
        h_lab = torch.empty(n, dtype=torch.int32).pin_memory()
        h_dst = torch.empty(n, dtype=torch.float32).pin_memory()
        d_fib = torch.empty_like(fib)

        def e2e_step():
            d_fib.copy_(h_fib, non_blocking=True)
            binding.seg_label(at, d_fib, args.mode, labels, dst, stream=stream)
            h_lab.copy_(labels, non_blocking=True)
            h_dst.copy_(dst, non_blocking=True)

        for _ in range(2):
            e2e_step()
        barrier()
        e0.record(stream)
        ke = max(1, min(args.steps, 5))
        for _ in range(ke):
            e2e_step()
        e1.record(stream)
        barrier()
        ems = e0.elapsed_time(e1) / ke
        t = torch.tensor([ems], device=dev, dtype=torch.float64)
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e = {"value": world * n / (float(t.item()) / 1000.0), "unit": UNIT,
               "h2d_bytes_per_step": int(h_fib.numel() * 4),
               "d2h_bytes_per_step": int(h_lab.numel() * 4 + h_dst.numel() * 4),
               "ms_per_step": float(t.item())}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    pk, pk_src = peaks()
    cpu = None
    pdpp = None
    if not args.no_cpu_baseline and world == 1:
        rate, n1, cores, pdpp, dt = oracle_sample_rate(atlas_np, fib_np, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n1} random fibers of the workload against all {atlas_np.M} "
                         f"centroids, FP64 progressive-discarding cascade (Section 2.3), "
                         f"{dt:.1f} s"}
    if pdpp is None:
        _, _, _, pdpp, _ = oracle_sample_rate(atlas_np, fib_np, 1.0)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    # FP32 CUDA-core peak: SMs x 128 lanes x 2 flop (FMA) x max SM clock
    peak_tf = sms * 128 * 2 * sm_max * 1e6 / 1e12
    alg_flop = n * atlas_np.M * pdpp * 8.0  # point distances of the paper's cascade x 8 flop
    if args.mode == "plain":
        achieved = alg_flop / (ms / 1000.0) / 1e12
        roof = {"bound": "alu", "kernel": "k_label_plain", "achieved": achieved, "peak": peak_tf,
                "unit": "TFLOP/s", "frac": achieved / peak_tf,
                "traffic": traffic_for("k_label_plain"),
                "peak_source": f"{sms} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz "
                               f"(max clock; {pk_src} clock)",
                "algorithmic": f"{pdpp:.4f} point distances per pair (oracle cascade counts) "
                               f"x 8 flop x {n} x {atlas_np.M} pairs"}
    else:
        roof = None
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "fibers": n, "centroids": atlas_np.M,
                       "bundles": atlas_np.B, "points": 21, "mode": args.mode,
                       "l2": "inputs larger than L2 (1.04 GB of fibers)",
                       "parallelism": f"dp{world} (fibers sharded by subject)"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": (launches_per_step * args.steps) if launches_per_step else None,
            "clocks": clk, "gemm_stats": stats, "context": PAPER_CONTEXT}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
