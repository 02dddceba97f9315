"""Workload descriptions (parameters only, no arithmetic of the method).

Sizes follow the paper's set-up (Table 1: two nested boxes, z = 0.1 - 1.5,
observer at the box centre, HEALPix Nside 1024) scaled to the benchmark
configurations below.  Lengths are in Mpc/h.
"""
from __future__ import annotations

from dataclasses import dataclass, field


@dataclass
class BoxSpec:
    L: float                 # side length
    n_side: int              # particles per side (n = n_side^3)
    sigma: float             # blob r.m.s. of the synthetic generator
    r_hi: float | None       # outer radius owned by this box (None: last shell edge)
    replicate: int = 0       # periodic image layers

    @property
    def n(self) -> int:
        return self.n_side ** 3


@dataclass
class Workload:
    name: str
    config: int
    boxes: list[BoxSpec]
    nside: int
    z_lo: float
    z_hi: float
    nshell: int
    spacing: str             # "dz": equal redshift steps, "dchi": equal comoving steps
    source: dict = field(default_factory=dict)
    omega_m: float = 0.3
    h: float = 0.7
    pdf_bins: int = 200


def tiny() -> Workload:
    """64^3 particles in a 500 Mpc/h periodic box, 10 equal-Delta-chi shells
    z = 0.1 - 0.5, single source plane z = 0.5, Nside 64."""
    return Workload("tiny_nside64", 1, [BoxSpec(500.0, 64, 5.0, None, replicate=4)],
                    64, 0.1, 0.5, 10, "dchi", dict(kind=0, z_s=0.5))


def nested(n_side: int = 512) -> Workload:
    """Two nested boxes (2000 and 6400 Mpc/h, n_side^3 particles each), the
    inner one owning r < 1000 Mpc/h, 40 shells z = 0.1 - 1.5, Nside 512."""
    return Workload("nested_nside512", 2,
                    [BoxSpec(2000.0, n_side, 5.0, 1000.0), BoxSpec(6400.0, n_side, 20.0, None)],
                    512, 0.1, 1.5, 40, "dz", dict(kind=0, z_s=1.5))


def full(n_side: int = 1024) -> Workload:
    """Full-size map: 2 x 1024^3 particles, 60 shells z = 0.1 - 1.5, Smail
    n(z) with alpha = 2, beta = 1.5, z0 = 0.5 on [0, 1.5], Nside 1024."""
    return Workload("full_nside1024", 3,
                    [BoxSpec(2000.0, n_side, 5.0, 1000.0), BoxSpec(6400.0, n_side, 20.0, None)],
                    1024, 0.1, 1.5, 60, "dz",
                    dict(kind=1, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5))


def batched(n_real: int = 150, n_side: int = 512) -> Workload:
    """Batched covariance: n_real realisations of the nested Nside-512 map,
    each box holding Poisson(f n_side^3) particles, f ~ U(0.5, 1.5)."""
    w = nested(n_side)
    w.name, w.config = "batched_nside512", 4
    w.source = dict(kind=1, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5)
    return w


WORKLOADS = {"tiny": tiny, "nested": nested, "full": full, "batched": batched}
