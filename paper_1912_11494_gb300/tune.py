"""Autotuner for the tile shapes of libseg's kernels (not in the paper).

Every mode has a few tile-shape configurations (seg_num_configs); all give identical results
and differ only in speed. tune() times each on a calibration slice of the caller's fibers with
CUDA events, selects the fastest on the atlas (seg_set_config) and caches the choice in a JSON
file keyed by device name, mode, atlas size and fiber-count bucket, so later processes reuse it.
"""
from __future__ import annotations

import json
import math
import os
import threading

import torch

from . import binding

_LOCK = threading.Lock()


def cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(base, "paper_1912_11494_gb300", "tuning.json")


def cache_key(device_name: str, mode: str, M: int, n: int) -> str:
    bucket = 1 << max(10, int(math.ceil(math.log2(max(n, 1)))))  # power-of-two fiber bucket
    return f"{device_name}|{mode}|M={M}|n<={bucket}"


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def time_config(atlas, fibers, mode: str, config: int, reps: int = 3) -> float:
    """Median milliseconds of one seg_label call with tile shape `config`."""
    binding.seg_set_config(atlas, mode, config)
    n = fibers.shape[0]
    labels = torch.empty(n, dtype=torch.int32, device=fibers.device)
    dist = torch.empty(n, dtype=torch.float32, device=fibers.device)
    binding.seg_label(atlas, fibers, mode, labels, dist)  # warm-up (and scratch growth)
    times = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        binding.seg_label(atlas, fibers, mode, labels, dist)
        e1.record()
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    binding.seg_sync_status(atlas)
    return sorted(times)[len(times) // 2]


def tune(atlas, fibers, mode: str = "plain", calib: int = 1 << 20, use_cache: bool = True,
         path: str | None = None) -> dict:
    """Select the fastest tile shape of `mode` for this atlas and fiber count; returns
    {"config": c, "ms": {c: t, ...}, "cached": bool}."""
    path = path or cache_path()
    dev_name = torch.cuda.get_device_name(fibers.device)
    key = cache_key(dev_name, mode, atlas.M, int(fibers.shape[0]))
    with _LOCK:
        data = _load(path) if use_cache else {}
        hit = data.get(key)
        if hit is not None and 0 <= hit["config"] < binding.seg_num_configs(mode):
            binding.seg_set_config(atlas, mode, hit["config"])
            return {"config": hit["config"], "ms": hit.get("ms", {}), "cached": True}
        sample = fibers[: min(int(fibers.shape[0]), calib)].contiguous()
        ms = {c: time_config(atlas, sample, mode, c)
              for c in range(binding.seg_num_configs(mode))}
        best = min(ms, key=ms.get)
        binding.seg_set_config(atlas, mode, best)
        if use_cache:
            data = _load(path)
            data[key] = {"config": best, "ms": {str(k): v for k, v in ms.items()}}
            _store(path, data)
        return {"config": best, "ms": ms, "cached": False}
