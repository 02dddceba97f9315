"""Seeded synthetic lightcone particles.

This module holds no arithmetic of the method itself: it only draws particle
positions, and serves both the CUDA library's callers and the oracle's tests.

Recipe (stand-in for the paper's L-PICOLA lightcone outputs, Table 1): a
fraction 0.7 of the particles is uniform in [0, L)^3; the other 0.3 sit in
isotropic Gaussian blobs of r.m.s. sigma around ``n_blob`` centres drawn
uniformly in the box, each particle picking its blob uniformly, positions
wrapped periodically.  Positions are drawn in FP64, rounded to FP32, and a
coordinate that rounds to L is set to 0, so every coordinate lies in [0, L).
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1801057450


def seed_for(config: int, realisation: int, box: int) -> int:
    """Seed of (config c, realisation r, box k): base + 1000 c + 10 r + k."""
    return SEED_BASE + 1000 * config + 10 * realisation + box


def particles_numpy(n: int, L: float, sigma: float, seed: int, n_blob: int = 1024,
                    blob_frac: float = 0.3) -> np.ndarray:
    """float32[n, 3] positions drawn with numpy's PCG64 generator (host)."""
    rng = np.random.default_rng(seed)
    centres = rng.random((n_blob, 3)) * L
    pos = rng.random((n, 3)) * L
    in_blob = rng.random(n) < blob_frac
    k = int(in_blob.sum())
    which = rng.integers(0, n_blob, size=k)
    off = rng.normal(size=(k, 3)) * sigma
    pos[in_blob] = np.mod(centres[which] + off, L)
    out = pos.astype(np.float32)
    out[out >= np.float32(L)] = 0.0
    return out


def particles_torch(n: int, L: float, sigma: float, seed: int, device="cuda",
                    n_blob: int = 1024, blob_frac: float = 0.3, chunk: int = 1 << 26,
                    out=None):
    """float32[n, 3] positions drawn on ``device`` with torch's generator.

    Drawn in chunks of ``chunk`` particles from one generator, so the result
    depends only on (n, L, sigma, seed, chunk).  ``out`` may be a
    preallocated float32 tensor of n*3 elements (it is filled and returned).
    """
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    if out is None:
        out = torch.empty((n, 3), dtype=torch.float32, device=device)
    out = out.view(-1, 3)
    centres = torch.rand((n_blob, 3), generator=g, device=device, dtype=torch.float64) * L
    Lf = torch.tensor(L, dtype=torch.float32, device=device)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        pos = torch.rand((m, 3), generator=g, device=device, dtype=torch.float64) * L
        in_blob = torch.rand((m,), generator=g, device=device, dtype=torch.float64) < blob_frac
        which = torch.randint(0, n_blob, (m,), generator=g, device=device)
        off = torch.randn((m, 3), generator=g, device=device, dtype=torch.float64) * sigma
        blob = torch.remainder(centres[which] + off, L)
        pos = torch.where(in_blob[:, None], blob, pos)
        p32 = pos.to(torch.float32)
        p32 = torch.where(p32 >= Lf, torch.zeros_like(p32), p32)
        out[s:s + m].copy_(p32)
        del pos, in_blob, which, off, blob, p32
    return out


def poisson_count(mean: float, seed: int) -> int:
    """Realisation size for the batched-covariance workload: f ~ U(0.5, 1.5),
    N ~ Poisson(f * mean)."""
    rng = np.random.default_rng(seed)
    f = rng.uniform(0.5, 1.5)
    return int(rng.poisson(f * mean))
