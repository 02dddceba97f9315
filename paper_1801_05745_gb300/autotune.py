"""Autotuner of the library's launch choices, by timing candidates once per
shape and caching the winner in a JSON file:
  - the binning output path (L2 atomics vs dense-key scatter with
    shared-memory histograms) per (GPU, Nside, shells, particle count);
  - the persistent batch kernel's particles per task and blocks per SM
    (ufc_set_tuning) per (GPU, Nside, shells, realisations, particle count).

Every choice gives identical results; only speed differs.  The cache lives in
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


_memo: dict = {}     # path -> (mtime, contents): the cache file is read once per change
_names: dict = {}    # device index -> GPU name


def _load() -> dict:
    p = cache_path()
    try:
        mt = os.path.getmtime(p)
    except OSError:
        return {}
    hit = _memo.get(p)
    if hit and hit[0] == mt:
        return dict(hit[1])
    try:
        with open(p) as f:
            d = json.load(f)
    except Exception:
        return {}
    _memo[p] = (mt, d)
    return dict(d)


def _gpu_name(device: int) -> str:
    if device not in _names:
        import torch
        _names[device] = torch.cuda.get_device_name(device)
    return _names[device]


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


def cached_bin_path(ctx, nside: int, nshell: int, n_total: int):
    """The cached binning path ('direct' or 'dense') for this shape, or None."""
    key = tune_key(_gpu_name(ctx.device), nside, nshell, n_total)
    with _lock:
        e = _load().get(key)
    return e["path"] if e else None


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


BATCH_CHUNKS = (2048, 8192, 32768)
BATCH_BLOCKS = (1, 2)


def batch_key(gpu_name: str, nside: int, nshell: int, nreal: int, n_total: int) -> str:
    nb = int(math.log2(max(1, n_total)))
    return f"batch|{gpu_name}|nside={nside}|nshell={nshell}|nreal={nreal}|log2n={nb}"


def cached_batch_tuning(ctx, nside: int, nshell: int, nreal: int, n_total: int):
    """The cached (batch_chunk, batch_blocks_per_sm) for this shape, or None."""
    key = batch_key(_gpu_name(ctx.device), nside, nshell, nreal, n_total)
    with _lock:
        e = _load().get(key)
    return (e["batch_chunk"], e["batch_blocks_per_sm"]) if e else None


def tune_batch(ctx, run, nside: int, nshell: int, nreal: int, n_total: int, reps: int = 2,
               force_retune: bool = False) -> dict:
    """Times run() (one batched call) under every candidate tuning of the
    persistent batch kernel, keeps the fastest in the context and the cache;
    returns {"batch_chunk", "batch_blocks_per_sm", "ms": {candidate: ms},
    "cached": bool}."""
    import torch
    key = batch_key(torch.cuda.get_device_name(ctx.device), nside, nshell, nreal, n_total)
    with _lock:
        e = _load().get(key)
    if e and not force_retune:
        ctx.set_tuning(e["batch_chunk"], e["batch_blocks_per_sm"])
        return dict(e, cached=True)
    times = {}
    for c in BATCH_CHUNKS:
        for b in BATCH_BLOCKS:
            ctx.set_tuning(c, b)
            run()                                  # warm-up (graph, workspace)
            torch.cuda.synchronize(ctx.device)
            s = torch.cuda.Event(enable_timing=True)
            t = torch.cuda.Event(enable_timing=True)
            s.record()
            for _ in range(reps):
                run()
            t.record()
            torch.cuda.synchronize(ctx.device)
            times[f"{c}x{b}"] = s.elapsed_time(t) / reps
    best = min(times, key=times.get)
    c, b = (int(v) for v in best.split("x"))
    ctx.set_tuning(c, b)
    entry = {"batch_chunk": c, "batch_blocks_per_sm": b, "ms": times}
    with _lock:
        cache = _load()
        cache[key] = entry
        _store(cache)
    return dict(entry, cached=False)
