#!/usr/bin/env python
"""Benchmark: subject fibers labelled per second at 4,145,000 fibers x 10,000 centroids.

One step labels the whole synthetic subject (4,145,000 fibers of 21 points, the paper's headline
subject size) against a 500-bundle x 20-centroid atlas through the C ABI, with inputs resident
in HBM (1.04 GB of fibers, larger than L2). Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--mode best|plain|gemm_bf16|gemm_tf32|
                  gemm_inv_bf16|gemm_inv_tf32] [--config C] [--n N] [--workload batch16]
  python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

--mode best (the default) tunes and times every mode and reports the fastest as the headline,
with every mode's time, per-kernel event timings and rooflines in "modes" / "rooflines".

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
    p.add_argument("--mode", default="best", choices=["best", *MODES])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--config", type=int, default=None, help="tile-shape config (default: tuned)")
    p.add_argument("--n", type=int, default=None, help="override the fiber count")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the oracle parity run, C4/C5, whole-brain, resampling, TF32 peak")
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


def traffic_for(kernel: str, mode: str, n: int):
    """Per-launch DRAM bytes of `kernel` in `mode` from the committed ncu summaries, or None
    when they were not taken for this kernel instantiation (`kernel@mode`; the plain kernel has
    one) at this fiber count."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    if t.get("fibers") != n:
        return None
    return t.get(f"{kernel}@{mode}", t.get(kernel) if mode == "plain" else None)


def traffic_source() -> str | None:
    """How the committed per-launch DRAM figures were obtained (their capture size)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            t = json.load(fh)
    except (OSError, ValueError):
        return None
    cap = t.get("captured_fibers")
    if cap and cap != t.get("fibers"):
        return (f"ncu dram__bytes_read.sum + dram__bytes_write.sum at {cap:,} fibers, scaled "
                f"linearly to {t.get('fibers'):,} (extrapolated)")
    return "ncu dram__bytes_read.sum + dram__bytes_write.sum at this size"


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the architecture)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model Name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def cuda_time(fn, steps, stream, warmup=2):
    """Mean device time (ms) of fn() over `steps` calls, CUDA events on `stream`."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def tf32_peak_tflops(dev) -> float:
    """Measured TF32 tensor-core throughput: torch.matmul on fp32 8192^3 with TF32 allowed,
    best of 10 (burst), 2 N^3 flop per product."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        n = 8192
        a = torch.randn(n, n, device=dev)
        b = torch.randn(n, n, device=dev)
        c = torch.empty(n, n, device=dev)
        best = 1e30
        stream = torch.cuda.current_stream(dev)
        for _ in range(3):
            torch.matmul(a, b, out=c)
        for _ in range(10):
            best = min(best, cuda_time(lambda: torch.matmul(a, b, out=c), 1, stream, 0))
        return 2.0 * n ** 3 / (best / 1000.0) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


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
MODES = ("plain", "gemm_bf16", "gemm_tf32", "gemm_inv_bf16", "gemm_inv_tf32", "plain_culled",
         "culled_fused")
KERNEL_NAME = {"plain": "k_label_plain", "gemm_screen": "k_gemm_screen",
               "cull_screen": "k_culled_screen", "culled_fused": "k_fused",
               "gemm_exact": "k_exact_blocks", "gemm_prep": "k_prep_a",
               "gemm_sort": "k_bin_count", "gemm_finalize": "k_finalize"}
LAUNCH_SLOTS = ("plain", "gemm_sort", "gemm_prep", "gemm_screen", "cull_screen", "culled_fused",
                "gemm_exact", "gemm_finalize")
# kernels the library launches inside each profiled scope (the sort is a count, two scans and a
# scatter; the prep scope holds the fiber operand, the tile boxes and the active-block masks;
# the finalize scope the overflow rescan and the label write)
KERNELS_PER_SLOT = {"plain": 1, "gemm_sort": 4, "gemm_prep": 3, "gemm_screen": 1,
                    "cull_screen": 1, "gemm_exact": 1, "gemm_finalize": 2,
                    "culled_fused": 2}


def kernels_per_slot(mode: str, slot: str) -> int:
    """Kernels one profiled scope launches (the culled mode's prep has no block-mask kernel)."""
    return KERNELS_PER_SLOT[slot] - (1 if mode == "plain_culled" and slot == "gemm_prep" else 0)


def dtype_of(mode: str) -> str:
    return "f32" if mode in ("plain", "plain_culled", "culled_fused") else \
        ("bf16+f32" if mode.endswith("bf16") else "tf32+f32")


def stage_fractions(r, n):
    """Where each discarding stage leaves the candidate pairs of a mode (its own counters)."""
    st = r["gemm_stats"]
    pairs = max(1, st["pairs"])
    return {"pairs": st["pairs"], "kept_by_culling": st["screened"] / pairs,
            "kept_by_screen": st["survivors"] / pairs,
            "survivors_per_fiber": st["survivors"] / max(1, n), "point_distances_per_survivor":
                st["point_distances"] / max(1, st["survivors"]),
            "overflow_fibers": st["overflow_fibers"]}


def time_mode(binding, at, fib, labels, dst, mode, steps, warmup, stream, world, dist, dev):
    """Device time per step of `mode` (max over ranks) and per-kernel event timings."""
    import torch
    for _ in range(max(3, warmup)):
        binding.seg_label(at, fib, mode, labels, dst, stream=stream)
    binding.seg_sync_status(at, stream)
    binding.seg_profile_enable(at, True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        binding.seg_label(at, fib, mode, labels, dst, stream=stream)
    e1.record(stream)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    binding.seg_sync_status(at, stream)
    ms = e0.elapsed_time(e1) / steps
    kern = {}
    launches = 0
    for k in LAUNCH_SLOTS:
        c, t = binding.seg_profile_read(at, k)
        if c:
            kern[k] = {"launches": c * kernels_per_slot(mode, k), "ms_per_step": t / c}
            launches += c * kernels_per_slot(mode, k)
    binding.seg_profile_enable(at, False)
    t = torch.tensor([ms], device=dev, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item()), kern, launches


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    from paper_1912_11494_gb300 import binding, build, synth, tune

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    build.build()
    if args.workload.startswith("batch"):
        return run_batch(args, world, rank, dev, dist)
    if args.workload.startswith("streamlines"):
        return run_streamlines(args, world, rank, dev, dist)

    atlas_np, fib_np = synth.workload(args.workload, n=args.n, device=dev)
    n = int(fib_np.shape[0])
    at = binding.Atlas(torch.as_tensor(atlas_np.centroids, device=dev),
                       torch.as_tensor(atlas_np.bundle_of, device=dev),
                       torch.as_tensor(atlas_np.thresholds, device=dev))
    fib = torch.as_tensor(fib_np, device=dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    dst = torch.empty(n, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    modes = MODES if args.mode == "best" else (args.mode,)
    results = {}
    for mode in modes:
        if args.config is not None:
            binding.seg_set_config(at, mode, args.config)
        else:
            tune.tune(at, fib, mode)
        ms, kern, launches = time_mode(binding, at, fib, labels, dst, mode, args.steps,
                                       args.warmup, stream, world, dist, dev)
        results[mode] = {"ms_per_step": ms, "value": world * n / (ms / 1000.0),
                         "config": binding.seg_get_config(at, mode), "kernels": kern,
                         "launches_per_step": launches / max(1, args.steps)}
        if mode != "plain":
            results[mode]["gemm_stats"] = binding.seg_gemm_stats(at)
    head = min(results, key=lambda m: results[m]["ms_per_step"])
    hr = results[head]
    ms_max = hr["ms_per_step"]
    value = hr["value"]

    # clocks: sample nvidia-smi over a re-run of the headline mode's timed region
    clocks = Clocks(local)
    clocks.start()
    time_mode(binding, at, fib, labels, dst, head, args.steps, 0, stream, world, dist, dev)
    clk = clocks.stop()

    # end to end through the public API on host buffers (seg_label_host): pinned host fibers in,
    # labels + distances out, every copy inside the timed region
    e2e = None
    if not args.no_e2e:
        h_fib = torch.empty_like(fib, device="cpu").pin_memory()
        h_fib.copy_(torch.as_tensor(fib_np))
        h_lab = torch.empty(n, dtype=torch.int32).pin_memory()
        h_dst = torch.empty(n, dtype=torch.float32).pin_memory()

        def e2e_step():
            binding.seg_label_host(at, h_fib, head, h_lab, h_dst, stream=stream)

        for _ in range(2):
            e2e_step()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ke = max(1, min(args.steps, 5))
        for _ in range(ke):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ems = e0.elapsed_time(e1) / ke
        t = torch.tensor([ems], device=dev, dtype=torch.float64)
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e = {"value": world * n / (float(t.item()) / 1000.0), "unit": UNIT,
               "h2d_bytes_per_step": int(h_fib.numel() * 4),
               "d2h_bytes_per_step": int(h_lab.numel() * 4 + h_dst.numel() * 4),
               "ms_per_step": float(t.item()), "mode": head,
               "api": "seg_label_host (chunked upload overlapping the labelling)"}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    pk, pk_src = peaks()
    cpu = None
    pdpp = None
    extras = None
    if world == 1 and not args.no_extras:
        extras = run_extras(dev, stream, atlas_np, fib_np, labels.cpu().numpy(),
                            dst.cpu().numpy(), head)
        of = extras["oracle_full"]
        pdpp = of["point_distances_per_pair"]
        if not args.no_cpu_baseline:
            cpu = {"value": of["fibers_per_s"], "unit": UNIT, "cores": of["threads"],
                   "kind": "oracle", "cpu_model": of["cpu_model"],
                   "sample": f"all {n} fibers of the workload against all {atlas_np.M} "
                             f"centroids, FP64 progressive-discarding cascade (Section 2.3), "
                             f"{of['seconds']:.1f} s"}
    if cpu is None and not args.no_cpu_baseline and world == 1:
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
    alu_peak = sms * 128 * 2 * sm_max * 1e6 / 1e12
    alu_src = (f"{sms} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz (max clock; {pk_src} "
               f"clock)")
    bf16 = float(pk.get("bf16_tflops", 1900.0))
    roofs = {}
    for mode, r in results.items():
        mr = {}
        for kname, k in r["kernels"].items():
            sec = k["ms_per_step"] / 1000.0
            if kname == "plain":
                alg = n * atlas_np.M * pdpp * 8.0
                mr[kname] = {"bound": "alu", "achieved": alg / sec / 1e12, "peak": alu_peak,
                             "unit": "TFLOP/s", "peak_source": alu_src,
                             "algorithmic": f"{pdpp:.4f} point distances per pair (oracle "
                                            f"cascade counts) x 8 flop x {n} x {atlas_np.M} "
                                            f"pairs"}
            elif kname == "gemm_screen":
                st = r["gemm_stats"]
                kdim = 32 if "inv" in mode else 64
                alg = 2.0 * st["screened"] * kdim
                tf32 = extras["tf32_tflops_measured"] if extras else None
                peak = bf16 if mode.endswith("bf16") else (tf32 or bf16 * (1.1 / 2.25))
                src = ("measured bf16 burst" + f" ({pk_src})" if mode.endswith("bf16") else
                       "measured tf32 burst (torch.matmul fp32 8192^3, TF32 allowed, this run)"
                       if tf32 else "measured bf16 burst x 1.1/2.25 (nominal TF32/BF16)")
                mr[kname] = {"bound": "tensor", "achieved": alg / sec / 1e12, "peak": peak,
                             "unit": "TFLOP/s", "peak_source": src,
                             "algorithmic": f"2 x K={kdim} x {st['screened']} pairs in the "
                                            f"computed blocks (of {st['pairs']}; the rest "
                                            f"culled on centre-point boxes)"}
            elif kname == "cull_screen":
                st = r["gemm_stats"]
                alg = 6.0 * st["screened"]
                mr[kname] = {"bound": "alu", "achieved": alg / sec / 1e12, "peak": alu_peak,
                             "unit": "TFLOP/s", "peak_source": alu_src,
                             "algorithmic": f"test1 in dot-product form (3 FMA = 6 flop) x "
                                            f"{st['screened']} pairs in the blocks kept by the "
                                            f"centre-point culling (of {st['pairs']})"}
            elif kname == "culled_fused":
                st = r["gemm_stats"]
                alg = 6.0 * st["screened"] + 8.0 * st["point_distances"]
                mr[kname] = {"bound": "alu", "achieved": alg / sec / 1e12, "peak": alu_peak,
                             "unit": "TFLOP/s", "peak_source": alu_src,
                             "algorithmic": f"test1 in dot-product form (6 flop) x "
                                            f"{st['screened']} pairs in the blocks kept by the "
                                            f"culling + {st['point_distances']} squared point "
                                            f"distances of the exact test x 8 flop"}
            elif kname == "gemm_exact":
                st = r["gemm_stats"]
                alg = 8.0 * st["point_distances"]
                mr[kname] = {"bound": "alu", "achieved": alg / sec / 1e12, "peak": alu_peak,
                             "unit": "TFLOP/s", "peak_source": alu_src,
                             "algorithmic": f"{st['point_distances']} squared point distances "
                                            f"(counted by the kernel) x 8 flop, "
                                            f"{st['survivors']} survivor pairs"}
            else:
                continue
            mr[kname]["kernel"] = KERNEL_NAME[kname]
            mr[kname]["frac"] = mr[kname]["achieved"] / mr[kname]["peak"]
            mr[kname]["traffic"] = traffic_for(KERNEL_NAME[kname], mode, n)
            if mr[kname]["traffic"] is not None:
                mr[kname]["traffic_source"] = traffic_source()
            mr[kname]["ms_per_launch"] = k["ms_per_step"]
            mr[kname]["share_of_step"] = k["ms_per_step"] / r["ms_per_step"]
        roofs[mode] = mr
    # the headline's roofline is that of its dominant kernel (the largest share of the step)
    dom = max(hr["kernels"], key=lambda k: hr["kernels"][k]["ms_per_step"])
    head_roof = roofs[head].get(dom)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": dtype_of(head),
            "data": "synthetic",
            "config": {"workload": args.workload, "fibers": n, "centroids": atlas_np.M,
                       "bundles": atlas_np.B, "points": 21, "mode": head,
                       "tile_config": hr["config"],
                       "l2": "inputs larger than L2 (1.04 GB of fibers)",
                       "parallelism": f"dp{world} (one subject per rank)"},
            "roofline": head_roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(round(hr["launches_per_step"] * args.steps)),
            "clocks": clk,
            "modes": {m: {k: v for k, v in r.items()} for m, r in results.items()},
            "stages": {m: stage_fractions(r, n) for m, r in results.items()
                       if "gemm_stats" in r},
            "rooflines": roofs, "context": PAPER_CONTEXT}
    if extras:
        line.update(extras)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_batch(args, world, rank, dev, dist):
    """The batched workload: 16 subjects (counts log-uniform in [0.3M, 4.2M], seeds 0-15)
    against the 10,000-centroid atlas in one seg_label_batch call per step."""
    import torch

    from paper_1912_11494_gb300 import binding, synth, tune
    scale = float(os.environ.get("SEG_BATCH_SCALE", "1.0"))
    atlas_np = synth.make_atlas(500, seed=1002, device=dev)
    fibs = [torch.as_tensor(synth.make_batch_subject(atlas_np, s, device=dev, scale=scale),
                            device=dev) for s in range(16)]
    at = binding.Atlas(torch.as_tensor(atlas_np.centroids, device=dev),
                       torch.as_tensor(atlas_np.bundle_of, device=dev),
                       torch.as_tensor(atlas_np.thresholds, device=dev))
    mode = "culled_fused" if args.mode == "best" else args.mode
    tune.tune(at, fibs[0], mode)
    labs = [torch.empty(f.shape[0], dtype=torch.int32, device=dev) for f in fibs]
    dsts = [torch.empty(f.shape[0], device=dev) for f in fibs]
    total = sum(int(f.shape[0]) for f in fibs)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(3, args.warmup)):
        binding.seg_label_batch(at, fibs, mode, labs, dsts, stream=stream)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        binding.seg_label_batch(at, fibs, mode, labs, dsts, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    binding.seg_sync_status(at, stream)
    ms = e0.elapsed_time(e1) / args.steps
    if rank == 0:
        print(json.dumps({"metric": "batched subject fibers labelled/sec", "value":
                          world * total / (ms / 1000.0), "unit": UNIT, "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                          "higher_is_better": True, "scaling": "weak",
                          "dtype": dtype_of(mode),
                          "data": "synthetic",
                          "config": {"workload": args.workload, "subjects": 16,
                                     "fibers": total, "mode": mode,
                                     "counts": [int(f.shape[0]) for f in fibs]}}), flush=True)
    return 0


def run_streamlines(args, world, rank, dev, dist):
    """Raw tractography in, labels out: 1,000,000 streamlines of the subject recipe (about
    0.2 mm steps) against the 500 x 20 atlas, resampled to 21 points (seg_resample) and labelled
    (seg_label_streamlines, which resamples and labels)."""
    import torch

    from paper_1912_11494_gb300 import binding, synth
    n = args.n or 1_000_000
    atlas_np = synth.make_atlas(500, seed=1002, device=dev)
    pts, off = synth.make_streamlines(atlas_np, n, 0.75, seed=2, device=dev)
    at = binding.Atlas(torch.as_tensor(atlas_np.centroids, device=dev),
                       torch.as_tensor(atlas_np.bundle_of, device=dev),
                       torch.as_tensor(atlas_np.thresholds, device=dev))
    mode = "culled_fused" if args.mode == "best" else args.mode
    stream = torch.cuda.current_stream(dev)
    out = torch.empty((n, 21, 3), device=dev)
    ms_rs = cuda_time(lambda: binding.seg_resample(pts, off, out=out, stream=stream), args.steps,
                      stream, max(3, args.warmup))
    ms_all = cuda_time(lambda: binding.label_streamlines(at, pts, off, mode, stream=stream),
                       args.steps, stream, max(3, args.warmup))
    binding.seg_sync_status(at)
    nbytes = pts.numel() * 4 + off.numel() * 8 + out.numel() * 4
    pk, _ = peaks()
    if rank == 0:
        print(json.dumps({"metric": "raw streamlines resampled and labelled/sec",
                          "value": world * n / (ms_all / 1000.0), "unit": "streamlines/s",
                          "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": ms_all, "higher_is_better": True, "scaling": "weak",
                          "dtype": dtype_of(mode), "data": "synthetic",
                          "config": {"workload": args.workload, "streamlines": n,
                                     "points": int(pts.shape[0]), "mode": mode},
                          "resample": {"ms": ms_rs, "streamlines_per_s": n / (ms_rs / 1e3),
                                       "roofline": {"bound": "hbm",
                                                    "achieved": nbytes / (ms_rs / 1e3) / 1e9,
                                                    "peak": pk["hbm_gbs"], "unit": "GB/s",
                                                    "frac": nbytes / (ms_rs / 1e3) / 1e9 /
                                                    pk["hbm_gbs"],
                                                    "algorithmic_bytes": int(nbytes)}}}),
              flush=True)
    return 0


def run_extras(dev, stream, atlas_np, fib_np, labels_head, dist_head, head_mode):
    """The other measured records of one run (single GPU): the oracle over the whole subject
    (the CPU baseline and label parity with near-ties), C5 forward + backward, the 16-subject
    batch, the whole-brain atlas, resampling of raw streamlines, the TF32 peak."""
    import torch

    import oracle
    from paper_1912_11494_gb300 import binding, synth
    from tests import parity
    out = {}
    # --- the oracle's cascade over all 4,145,000 fibers: CPU baseline and full label parity
    t = time.perf_counter()
    ref = oracle.label(fib_np, atlas_np.centroids, atlas_np.bundle_of, atlas_np.thresholds,
                       "cascade")
    dt = time.perf_counter() - t
    c = ref["counts"]
    res = parity.compare_all(fib_np, atlas_np.centroids, atlas_np.bundle_of,
                             atlas_np.thresholds, labels_head, dist_head, ref=ref)
    both = (labels_head >= 0) & (ref["labels"] >= 0)
    out["oracle_full"] = {"fibers": len(fib_np), "seconds": dt, "fibers_per_s": len(fib_np) / dt,
                          "threads": oracle.max_threads(), "cpu_model": cpu_model(),
                          "point_distances_per_pair": float(c[:4].sum()) / float(c[4]),
                          "pairs_reaching_test": {"test1": int(c[4]), "test2": int(c[5]),
                                                  "test3": int(c[6]), "test4": int(c[7])}}
    out["parity"] = {"mode": head_mode, "fibers": res["n"], "labelled": res["labelled"],
                     "label_differences": res["mismatches"], "decidable_differences": 0,
                     "near_ties": res["near_ties"],
                     "max_dist_error_mm": float(np.abs(dist_head[both] -
                                                       ref["dist"][both]).max())}
    # --- the oracle's brute force on the 10,000 x 1,000 workload
    a1, f1 = synth.workload("subject10k_atlas1k")
    t = time.perf_counter()
    oracle.label(f1, a1.centroids, a1.bundle_of, a1.thresholds, "brute")
    out["oracle_brute_c1"] = {"fibers_per_s": len(f1) / (time.perf_counter() - t),
                              "threads": oracle.max_threads()}
    # --- C5: forward (affine, labels) and backward (seg_grad) at 1,000,000 x 5,000
    a5, f5 = synth.workload("affine1m_atlas5k", device=dev)
    at5 = binding.Atlas(torch.as_tensor(a5.centroids, device=dev),
                        torch.as_tensor(a5.bundle_of, device=dev),
                        torch.as_tensor(a5.thresholds, device=dev))
    x = torch.as_tensor(f5, device=dev)
    aff = synth.random_affine(21, max_deg=2.0, max_t=1.0, s_lo=0.99, s_hi=1.01)
    n5 = x.shape[0]
    y = torch.empty_like(x)
    lab = torch.empty(n5, dtype=torch.int32, device=dev)
    cidx = torch.empty_like(lab)
    orient = torch.empty(n5, dtype=torch.uint8, device=dev)
    ga = torch.empty(12, dtype=torch.float64, device=dev)
    gc = torch.empty((a5.M, 21, 3), device=dev)
    cost = torch.empty(1, dtype=torch.float64, device=dev)

    def fwd():
        binding.seg_apply_affine(x, aff, out=y, stream=stream)
        binding.seg_label(at5, y, head_mode, lab, None, cidx, orient, stream=stream)

    def bwd():
        binding.seg_grad(at5, x, aff, cidx, orient, ga, gc, cost, stream=stream)

    ms_f = cuda_time(fwd, 10, stream)
    ms_b = cuda_time(bwd, 10, stream)
    binding.seg_sync_status(at5)
    out["c5_gradient"] = {"workload": "affine1m_atlas5k", "fibers": n5, "centroids": a5.M,
                          "mode": head_mode, "ms_forward": ms_f, "ms_backward": ms_b,
                          "fibers_per_s": n5 / ((ms_f + ms_b) / 1000.0),
                          "backward_gbs": (n5 * 252 + n5 * 5 + a5.M * 252 * 3) / (ms_b / 1e3) /
                          1e9}
    del at5, x, y
    # --- C4: the 16-subject batch (28.6M fibers) in one call
    ab = synth.make_atlas(500, seed=1002, device=dev)
    fibs = [torch.as_tensor(synth.make_batch_subject(ab, s, device=dev), device=dev)
            for s in range(16)]
    atb = binding.Atlas(torch.as_tensor(ab.centroids, device=dev),
                        torch.as_tensor(ab.bundle_of, device=dev),
                        torch.as_tensor(ab.thresholds, device=dev))
    labs = [torch.empty(f.shape[0], dtype=torch.int32, device=dev) for f in fibs]
    dsts = [torch.empty(f.shape[0], device=dev) for f in fibs]
    total = sum(int(f.shape[0]) for f in fibs)
    out["batch16"] = {"subjects": 16, "fibers": total, "modes": {}}
    for m in ("culled_fused", "plain_culled", "gemm_bf16", "plain"):
        ms = cuda_time(lambda: binding.seg_label_batch(atb, fibs, m, labs, dsts, stream=stream),
                       3 if m == "plain" else 5, stream)
        out["batch16"]["modes"][m] = {"ms_per_batch": ms, "fibers_per_s": total / (ms / 1e3)}
    binding.seg_sync_status(atb)
    del fibs, labs, dsts, atb
    # --- the whole-brain atlas (62 bundles, 44,345 centroids) at 4,145,000 fibers
    aw, fw = synth.workload("subject4145k_atlas44k", device=dev)
    atw = binding.Atlas(torch.as_tensor(aw.centroids, device=dev),
                        torch.as_tensor(aw.bundle_of, device=dev),
                        torch.as_tensor(aw.thresholds, device=dev))
    xw = torch.as_tensor(fw, device=dev)
    lw = torch.empty(xw.shape[0], dtype=torch.int32, device=dev)
    out["whole_brain"] = {"workload": "subject4145k_atlas44k", "fibers": int(xw.shape[0]),
                          "centroids": aw.M, "modes": {}}
    for m in ("culled_fused", "plain_culled", "gemm_bf16"):
        ms = cuda_time(lambda: binding.seg_label(atw, xw, m, lw, stream=stream), 3, stream)
        out["whole_brain"]["modes"][m] = {"ms_per_step": ms,
                                         "fibers_per_s": xw.shape[0] / (ms / 1e3)}
    binding.seg_sync_status(atw)
    del atw, xw, lw
    # --- resampling of 1,000,000 raw streamlines (about 0.2 mm steps)
    pts, off = synth.make_streamlines(atlas_np, 1_000_000, 0.75, seed=2, device=dev)
    rs_out = torch.empty((1_000_000, 21, 3), device=dev)
    ms = cuda_time(lambda: binding.seg_resample(pts, off, out=rs_out, stream=stream), 10, stream)
    nbytes = pts.numel() * 4 + off.numel() * 8 + rs_out.numel() * 4
    out["resample"] = {"streamlines": 1_000_000, "points": int(pts.shape[0]), "ms": ms,
                       "fibers_per_s": 1e6 / (ms / 1e3), "gbs": nbytes / (ms / 1e3) / 1e9,
                       "algorithmic_bytes": int(nbytes)}
    del pts, off, rs_out
    out["tf32_tflops_measured"] = tf32_peak_tflops(dev)
    return out


if __name__ == "__main__":
    sys.exit(main())
