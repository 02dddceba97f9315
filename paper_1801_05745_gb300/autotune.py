"""Choice of the binning output path (L2 atomics vs dense-key scatter with
shared-memory histograms) by timing both once per (GPU, Nside, shells,
particle count) and caching the winner in a JSON file.

Both paths give identical count maps; only speed differs.  The cache lives in
$UFC_AUTOTUNE_CACHE, else ~/.cache/ufalcon_gb300/autotune.json.
"""
from __future__ import annotations

import json
import math
import os
import threading

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("UFC_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "ufalcon_gb300",
                                       "autotune.json"))


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(d: dict) -> None:
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def tune_key(gpu_name: str, nside: int, nshell: int, n_total: int) -> str:
    """Particle counts are bucketed by powers of 2."""
    nb = int(math.log2(max(1, n_total)))
    return f"{gpu_name}|nside={nside}|nshell={nshell}|log2n={nb}"


def choose_bin_path(ctx, xyz_list, boxes, chi_edges, nside: int, counts=None, reps: int = 2,
                    force_retune: bool = False) -> str:
    """'direct' or 'dense' for this binning call shape (times both once)."""
    import torch
    gpu = torch.cuda.get_device_name(ctx.device)
    n_total = sum(x.numel() // 3 for x in xyz_list)
    key = tune_key(gpu, nside, len(chi_edges) - 1, n_total)
    with _lock:
        cache = _load()
        if key in cache and not force_retune:
            return cache[key]["path"]
    times = {}
    for path in ("direct", "dense"):
        try:
            counts = ctx.bin(xyz_list, boxes, chi_edges, nside, counts=counts, path=path)
        except Exception:
            continue                      # path not available for this shape
        torch.cuda.synchronize(ctx.device)
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        for _ in range(reps):
            ctx.bin(xyz_list, boxes, chi_edges, nside, counts=counts, path=path)
        e.record()
        torch.cuda.synchronize(ctx.device)
        times[path] = s.elapsed_time(e) / reps
    best = min(times, key=times.get)
    with _lock:
        cache = _load()
        cache[key] = {"path": best, "ms": times}
        _store(cache)
    return best
