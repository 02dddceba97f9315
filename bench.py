#!/usr/bin/env python
"""Benchmark of the GB300 lightcone hot path.

One step = one realisation of the full-size map, the whole hot path:
  bin 2 x 1024^3 particles of two nested boxes into 60 shells x Nside 1024
  (Eq. 5, 8), kappa map + moments + PDF (Eq. 6, 12-13) and the adjoint
  d(var, skew)/d theta in one read of the counts, statistics vector and
  FP64 Welford covariance update (Eq. 10).
The shell weights are per-cosmology constants computed once before timing.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line (rank 0).  Under torchrun each rank bins its own
realisation (weak scaling, no data-path collective).  --impl reference times
the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("G particles/s binned and kappa maps/s at Nside 1024 (% HBM roofline); "
          "batched vs serial")
UNIT = "Gparticles/s"
PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# DRAM bytes (read + write) per particle of the fast stage, from an ncu
# capture of k_fast_tma on two boxes of 512^3 particles at Nside 512 (two
# launches of 134.2M particles: 1.868 and 1.838 GB); scaled to a launch by
# its particle count.  Retake it whenever k_fast_tma changes.
FAST_TRAFFIC_PER_PARTICLE = (1.610987e9 + 257.307648e6 + 1.611105e9 + 227.374336e6) / 2 / 134217728
# DRAM bytes of every binning kernel above the algorithmic ones (particles
# read, count maps written), per keyed particle: ncu dram__bytes_read+write
# of one binning call of two boxes of 512^3 particles at Nside 1024, 60
# shells (8.802 GB measured, 6.241 GB algorithmic, 125.0M keyed particles)
BIN_SCRATCH_PER_KEY = (4.695745792e9 + 4.106062848e9 - 6.241124352e9) / 125014670


def hbm_peak():
    try:
        with open(PEAKS) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload(scale_side: int | None):
    from paper_1801_05745_gb300 import workloads
    w = workloads.full() if scale_side is None else workloads.full(scale_side)
    return w


def shells(w, api=None, orc=None):
    z = np.linspace(w.z_lo, w.z_hi, w.nshell + 1)
    if api is not None:
        chi = api.chi_edges(api.make_cosmo(w.omega_m, w.h, 1), z)
    else:
        chi = orc.chi_edges(w.omega_m, w.h, 1, z)
    split = int(np.argmin(np.abs(chi - w.boxes[0].r_hi)))
    return z, chi, split


# ----------------------------------------------------------------- clocks ----
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i]
                          and "Not" not in r[5 + i]})
        loaded = [v for v in sm if v > 0.5 * mx] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


# ----------------------------------------------------------- CPU baseline ----
def cpu_baseline(w, parts_host, counts_host, A, C, dAC, seconds_budget=20.0):
    """The oracle, as it stands, on a bounded sample of the workload:
    binning of a particle sample, one full kappa map with moments and PDF,
    and the complex-step gradient on a map of 1/16 the pixels (scaled)."""
    import oracle
    oracle.build()
    z, chi, split = shells(w, orc=oracle)
    boxes = [oracle.make_box(2000.0, [1000.0] * 3, w.boxes[0].n, 0, split),
             oracle.make_box(6400.0, [3200.0] * 3, w.boxes[1].n, split, w.nshell)]
    n_total = sum(b.n for b in w.boxes)
    # binning sample: grow until ~40% of the budget
    m = 1 << 18
    t_bin = 0.0
    done = 0
    while True:
        t0 = time.perf_counter()
        for k in range(2):
            oracle.keys(parts_host[k][:m], boxes[k], chi, w.nside)
        t = time.perf_counter() - t0
        t_bin, done = t, 2 * m
        if t > 0.4 * seconds_budget or m >= len(parts_host[0]):
            break
        m = min(len(parts_host[0]), m * 4)
    per_particle = t_bin / done
    t0 = time.perf_counter()
    kap = oracle.kappa_map(counts_host, A, C)
    t_kappa = time.perf_counter() - t0
    t0 = time.perf_counter()
    mom = oracle.moments(kap)
    oracle.pdf(kap, mom[0] - 6 * mom[1] ** 0.5, mom[0] + 6 * mom[1] ** 0.5, w.pdf_bins)
    t_stats = time.perf_counter() - t0
    # adjoint on a quarter-resolution map (1/16 of the pixels), scaled by 16
    sub = counts_host.reshape(w.nshell, -1)[:, : counts_host.shape[1] // 16]
    nside_sub = w.nside // 4
    src = oracle.make_source(kind=1, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5)
    t0 = time.perf_counter()
    oracle.kappa_stat_grads(np.ascontiguousarray(sub), nside_sub, w.omega_m, w.h, 1, boxes, z, src)
    t_grad = (time.perf_counter() - t0) * 16
    t_step = per_particle * n_total + t_kappa + t_stats + t_grad
    # the oracle's OpenMP binning (all host cores, atomic increments) on the
    # same sample, the rest of the step as above
    counts_omp = np.zeros((w.nshell, 12 * w.nside ** 2), dtype=np.int32)
    counts_omp.fill(0)              # touch every page before the timed region
    t0 = time.perf_counter()
    threads = 1
    for k in range(2):
        _, _, threads = oracle.bin_counts_omp(parts_host[k][:m], boxes[k], chi, w.nside, counts_omp)
    per_particle_omp = (time.perf_counter() - t0) / done
    del counts_omp
    t_step_omp = per_particle_omp * n_total + t_kappa + t_stats + t_grad
    return {
        "value": n_total / t_step / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
        "sample": (f"oracle keys of {done} particles ({per_particle * 1e9:.0f} ns each, scaled to "
                   f"{n_total}); one full Nside {w.nside} kappa map {t_kappa:.2f} s; moments+PDF "
                   f"{t_stats:.2f} s; complex-step gradient on 1/16 of the pixels x16 = "
                   f"{t_grad:.1f} s; estimated {t_step:.1f} s per step, single thread"),
        "all_cores": {
            "value": n_total / t_step_omp / 1e9, "unit": UNIT, "cores": threads,
            "kind": "oracle (OpenMP binning)",
            "sample": (f"oracle OpenMP binning of the same {done} particles on {threads} threads "
                       f"({per_particle_omp * 1e9:.1f} ns each, scaled to {n_total}); kappa map, "
                       f"moments, PDF and gradient single-threaded as above; estimated "
                       f"{t_step_omp:.1f} s per step"),
            "binning_gparticles_per_s": 1e-9 / per_particle_omp,
        },
    }


# ------------------------------------------------- batched vs serial leg ----
def batched_leg(ctx, api, synth, dev, n_real: int, n_side: int, nbuf: int = 8,
                nside: int | None = None):
    """Covariance of n_real realisations of the nested Nside-512 map, each box
    holding Poisson(f n_side^3) particles, f ~ U(0.5, 1.5): one graph-captured
    ufc_batched_stats call against the same maps one at a time through
    ufc_bin + ufc_kappa_stats + ufc_stats_vector + ufc_welford_update.

    Positions come from nbuf seeded buffers per box, 1.5 n_side^3 (+6 sigma)
    particles each; realisation r takes its own seeded count and a seeded
    48-byte-aligned start inside buffer r mod nbuf, so every realisation is a
    different particle set of its drawn size."""
    import torch
    from paper_1801_05745_gb300 import workloads
    wb = workloads.batched(n_real, n_side)
    if nside is not None:
        wb.nside = nside
        wb.name = f"batched_nside{nside}"
    z, chi, split = shells(wb, api=api)
    cosmo = api.make_cosmo(wb.omega_m, wb.h, 1)
    src = api.make_source(kind=1, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5)
    mean = wb.boxes[0].n
    cap = int(1.5 * mean + 6 * (1.5 * mean) ** 0.5) + 8
    bufs = [[synth.particles_torch(cap, wb.boxes[k].L, wb.boxes[k].sigma,
                                   synth.seed_for(4, 1000 + i, k), device=dev) for k in range(2)]
            for i in range(nbuf)]
    obs = [[1000.0] * 3, [3200.0] * 3]
    rng = np.random.default_rng(synth.seed_for(4, 999, 0))
    xyz, boxes, A, C, n_tot = [], [], [], [], 0
    for r in range(n_real):
        row, brow = [], []
        for k in range(2):
            n_rk = min(synth.poisson_count(mean, synth.seed_for(4, r, k)), cap)
            o = 4 * int(rng.integers(0, (cap - n_rk) // 4 + 1))
            row.append(bufs[r % nbuf][k][o:o + n_rk])
            lo_, hi_ = (0, split) if k == 0 else (split, wb.nshell)
            brow.append(api.make_box(wb.boxes[k].L, obs[k], n_rk, lo_, hi_))
            n_tot += n_rk
        a, _, c = api.kappa_coeffs(cosmo, brow, z, wb.nside, src)
        xyz.append(row)
        boxes.append(brow)
        A.append(a)
        C.append(c)
    A, C = np.array(A), np.array(C)
    npix = 12 * wb.nside ** 2
    counts = torch.empty((wb.nshell, npix), dtype=torch.int32, device=dev)
    kap = torch.empty(npix, dtype=torch.float32, device=dev)
    nb = wb.pdf_bins
    d = 6 + nb
    ctx.reserve(wb.nside, wb.nshell, max(x.shape[0] for row in xyz for x in row))
    ctx.bin(xyz[0], boxes[0], chi, wb.nside, counts=counts)
    _, m0, _ = ctx.kappa_stats(counts, A[0], C[0], -1.0, 1.0, nb, kappa=kap)
    m0 = m0.cpu().numpy()
    lo, hi = float(m0[0] - 6 * m0[1] ** 0.5), float(m0[0] + 6 * m0[1] ** 0.5)
    vec = torch.empty(d, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def serial(state):
        for r in range(n_real):
            ctx.bin(xyz[r], boxes[r], chi, wb.nside, counts=counts)
            _, mom, pdf = ctx.kappa_stats(counts, A[r], C[r], lo, hi, nb, kappa=kap)
            ctx.stats_vector(mom, pdf, out=vec)
            ctx.welford_update(vec.view(1, d), state)

    def batched(state):
        ctx.batched_stats(xyz, boxes, chi, wb.nside, A, C, lo, hi, nb, state, graph=True,
                          counts=counts, kappa=kap)

    def batched_launches(state):
        ctx.batched_stats(xyz, boxes, chi, wb.nside, A, C, lo, hi, nb, state, graph=True,
                          counts=counts, kappa=kap, launches=True)

    from paper_1801_05745_gb300 import autotune
    tsc = api.welford_state(d, dev)
    tuning = autotune.tune_batch(ctx, lambda: batched(tsc), wb.nside, wb.nshell, n_real, n_tot)
    out = {}
    states = {}
    for name, fn_ in (("serial", serial), ("batched", batched),
                      ("batched_launches", batched_launches)):
        fn_(api.welford_state(d, dev))             # warm-up (graph instantiation, workspace)
        st = api.welford_state(d, dev)
        torch.cuda.synchronize()
        e0.record(stream)
        fn_(st)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = {"ms": ms, "maps_per_s": n_real / (ms * 1e-3),
                     "gparticles_per_s": n_tot / (ms * 1e-3) / 1e9}
        states[name] = st
    out["states_equal"] = bool(torch.equal(states["serial"], states["batched"]) and
                               torch.equal(states["serial"], states["batched_launches"]))
    out["speedup"] = out["serial"]["ms"] / out["batched"]["ms"]
    out["speedup_launches"] = out["serial"]["ms"] / out["batched_launches"]["ms"]
    out["tuning"] = {k: tuning[k] for k in ("batch_chunk", "batch_blocks_per_sm", "cached")}
    out["tuning"]["candidates_ms"] = tuning.get("ms")
    # GPU time per kernel of the serial run (a separate, profiled pass) and of
    # the batched call's persistent kernel outside a graph
    ctx.profile(True)
    serial(api.welford_state(d, dev))
    torch.cuda.synchronize()
    out["serial_kernels_ms"] = {k: round(v[0], 3) for k, v in ctx.profile_read().items()}
    ctx.batched_stats(xyz, boxes, chi, wb.nside, A, C, lo, hi, nb, api.welford_state(d, dev),
                      graph=False, counts=counts, kappa=kap)
    torch.cuda.synchronize()
    out["batched_kernels_ms"] = {k: round(v[0], 3) for k, v in ctx.profile_read().items()}
    ctx.profile(False)
    out["config"] = {"workload": wb.name, "realisations": n_real, "nside": wb.nside,
                     "nshell": wb.nshell, "particles": n_tot,
                     "per_box": f"Poisson(f {n_side}^3), f ~ U(0.5, 1.5)",
                     "position_buffers": nbuf}
    del bufs, xyz
    return out


def snapshot_leg(ctx, api, synth, dev, w, z, chi, n_per: int = 1 << 25):
    """Snapshot-mode lightcone (ufc_bin_snapshots): one snapshot at every
    second shell edge (30 for 60 shells, each filling two shells), each of
    n_per particles in a 6400 Mpc/h box around the observer, Nside of the
    workload.  Every snapshot is read once per call; the rate counts all of
    their particles."""
    import torch
    z_snap = z[:-1:2]
    sos = api.snapshot_assign(z, z_snap)
    xs = [synth.particles_torch(n_per, 6400.0, w.boxes[1].sigma, synth.seed_for(5, s, 1),
                                device=dev) for s in range(len(z_snap))]
    geoms = [api.make_box(6400.0, [3200.0] * 3, n_per, 0, 1) for _ in xs]
    counts = torch.empty((w.nshell, 12 * w.nside ** 2), dtype=torch.int32, device=dev)
    ctx.bin_snapshots(xs, geoms, sos, chi, w.nside, counts=counts)      # warm-up
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    reps = 3
    torch.cuda.synchronize()
    ctx.profile(True)
    e0.record(stream)
    for _ in range(reps):
        ctx.bin_snapshots(xs, geoms, sos, chi, w.nside, counts=counts)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    ms = e0.elapsed_time(e1) / reps
    n_tot = n_per * len(xs)
    info = ctx.bin_info()
    fast_ms = prof.get("k_fast", (0.0, 1))[0] / reps
    out = {"ms": ms, "gparticles_per_s": n_tot / (ms * 1e-3) / 1e9,
           "k_fast_ms": fast_ms,
           "k_fast_frac_of_peak": (12.0 * n_tot / (fast_ms * 1e-3) / 1e9) / hbm_peak()[0]
           if fast_ms else None,
           "kernels_ms": {k: round(v[0] / reps, 3) for k, v in prof.items()},
           "in_shells_last_pass": info["keyed"],
           "config": {"workload": "snapshots_nside%d" % w.nside, "snapshots": len(xs),
                      "particles_per_snapshot": n_per, "box": "6400 Mpc/h",
                      "nshell": w.nshell, "nside": w.nside,
                      "shells_per_snapshot": 2}}
    del xs
    return out


# ---------------------------------------------------------- reference arm ----
def run_reference(args):
    """The oracle as the reference arm: each step bins a bounded particle
    sample of the workload and builds one full kappa map with statistics."""
    import oracle
    from paper_1801_05745_gb300 import synth
    oracle.build()
    w = workload(args.scale)
    if args.nside:
        w.nside = args.nside
    z, chi, split = shells(w, orc=oracle)
    boxes = [oracle.make_box(2000.0, [1000.0] * 3, w.boxes[0].n, 0, split),
             oracle.make_box(6400.0, [3200.0] * 3, w.boxes[1].n, split, w.nshell)]
    src = oracle.make_source(kind=1, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5)
    A, B, C = oracle.kappa_coeffs(w.omega_m, w.h, 1, boxes, z, w.nside, src)
    m = args.ref_sample
    n_total = sum(b.n for b in w.boxes)
    times = []
    for step in range(args.warmup + args.steps):
        parts = [synth.particles_numpy(m, 2000.0, 5.0, synth.seed_for(3, step, 0)),
                 synth.particles_numpy(m, 6400.0, 20.0, synth.seed_for(3, step, 1))]
        counts = np.zeros((w.nshell, 12 * w.nside ** 2), np.int32)
        t0 = time.perf_counter()
        for k in range(2):
            oracle.bin_counts(parts[k], boxes[k], chi, w.nside, counts)
        t_bin = time.perf_counter() - t0
        t0 = time.perf_counter()
        kap = oracle.kappa_map(counts, A, C)
        mom = oracle.moments(kap)
        oracle.pdf(kap, -0.05, 0.2, w.pdf_bins)
        t_map = time.perf_counter() - t0
        est = t_bin / (2 * m) * n_total + t_map
        if step >= args.warmup:
            times.append(est)
    t = float(np.mean(times))
    val = n_total / t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "particles": n_total, "nside": w.nside, "nshell": w.nshell},
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"per-step time EXTRAPOLATED: {2 * m} particles binned per "
                                   f"step, their time scaled linearly to {n_total} particles, plus "
                                   f"one full Nside {w.nside} kappa map, moments and PDF (timed "
                                   f"whole); single thread"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ main ----
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--scale", type=int, default=None, help="particles per side per box (default 1024)")
    ap.add_argument("--nside", type=int, default=None, help="HEALPix Nside (default 1024)")
    ap.add_argument("--ref-sample", type=int, default=1_000_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-cl", action="store_true")
    ap.add_argument("--no-snapshots", action="store_true")
    ap.add_argument("--batched-real", type=int, default=150)
    ap.add_argument("--batched-side", type=int, default=512)
    ap.add_argument("--nshell", type=int, default=None, help="shells (default 60)")
    ap.add_argument("--path", default=None, choices=["direct", "dense"],
                    help="force the binning output path (default: the library's choice)")
    ap.add_argument("--split", default="realisation", choices=["realisation", "subvolume"],
                    help="multi-GPU decomposition: each rank its own realisation (weak "
                         "scaling), or each rank a shard of every box, the FP64 partial kappa "
                         "sums and the adjoint's per-shell sums all-reduced inside the step "
                         "(Sec. 2.4; strong)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1801_05745_gb300 import build as pbuild
    pbuild.build()
    from paper_1801_05745_gb300 import api, synth

    w = workload(args.scale)
    if args.nside:
        w.nside = args.nside
    if args.nshell:
        w.nshell = args.nshell
    sub = args.split == "subvolume"
    ctx = api.context(local)
    cosmo = api.make_cosmo(w.omega_m, w.h, 1)
    z, chi, split = shells(w, api=api)
    boxes = [api.make_box(2000.0, [1000.0] * 3, w.boxes[0].n, 0, split),
             api.make_box(6400.0, [3200.0] * 3, w.boxes[1].n, split, w.nshell)]
    src = api.make_source(kind=1, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5)
    A, B, C, dA, dC = api.kappa_coeffs(cosmo, boxes, z, w.nside, src, derivs=True)
    n_total = sum(b.n for b in w.boxes)

    dev = torch.device("cuda", local)
    # realisation split: rank r draws realisation r; subvolume split: every
    # rank draws realisation 0 and keeps its shard of each box (shard starts
    # on multiples of 4 particles, so that the bulk copies stay aligned)
    parts = [synth.particles_torch(w.boxes[k].n, w.boxes[k].L, w.boxes[k].sigma,
                                   synth.seed_for(3, 0 if sub else rank, k), device=dev)
             for k in range(2)]
    if sub:
        from paper_1801_05745_gb300 import parallel
        parts = [p[slice(*parallel.shard_range(p.shape[0], rank, world, align=4))] for p in parts]
    n_local = sum(p.shape[0] for p in parts)
    npix = 12 * w.nside ** 2
    counts = torch.empty((w.nshell, npix), dtype=torch.int32, device=dev)
    kap = torch.empty(npix, dtype=torch.float32, device=dev)
    d = 6 + w.pdf_bins
    wstate = api.welford_state(d, dev)
    vec = torch.empty(d, dtype=torch.float64, device=dev)
    ctx.reserve(w.nside, w.nshell, max(b.n for b in w.boxes))
    # subvolume split: the ranks' FP64 partial kappa sums (8 B per pixel) and
    # the adjoint's per-shell sums are all-reduced, not the count maps
    partial = torch.empty(npix, dtype=torch.float64, device=dev) if sub else None

    # binning path: the autotuner's choice for this shape (timed once, cached),
    # unless --path forces one
    from paper_1801_05745_gb300 import autotune
    bin_path = args.path or autotune.choose_bin_path(ctx, parts, boxes, chi, w.nside, counts=counts)
    # PDF range from a first map: mean +- 6 sigma, then fixed
    ctx.bin(parts, boxes, chi, w.nside, counts=counts, path=bin_path)
    if sub:
        _, mom, _ = parallel.subvolume_kappa(ctx, counts, A, C, -1.0, 1.0, w.pdf_bins, kappa=kap,
                                             partial=partial)
    else:
        _, mom, _ = ctx.kappa_stats(counts, A, C, -1.0, 1.0, w.pdf_bins, kappa=kap)
    m0 = mom.cpu().numpy()
    lo, hi = float(m0[0] - 6 * m0[1] ** 0.5), float(m0[0] + 6 * m0[1] ** 0.5)

    nvtx = torch.cuda.nvtx

    def step(host=None):
        # NVTX ranges of the step's phases (the library adds one per kernel)
        nvtx.range_push("bin")
        if host is None:
            ctx.bin(parts, boxes, chi, w.nside, counts=counts, path=bin_path)
        else:                                    # host buffers through ufc_bin_host
            ctx.bin_host(host, boxes, chi, w.nside, counts=counts, path=bin_path)
        nvtx.range_pop()
        # kappa map, moments, PDF and the adjoint of var + skew in one read of
        # the counts (ufc_kappa_stats_backward; with the subvolume split the
        # partial sums' all-reduce first, then ufc_kappa_adjoint_sums and the
        # per-shell sums' all-reduce), then the covariance update
        nvtx.range_push("kappa_stats_adjoint")
        if sub:
            _, mom, pdf, grad, _, _ = parallel.subvolume_kappa(
                ctx, counts, A, C, lo, hi, w.pdf_bins, dA=dA, dC=dC, w_var=1.0, w_skew=1.0,
                kappa=kap, partial=partial)
        else:
            _, mom, pdf, grad, _, _ = ctx.kappa_stats_backward(counts, A, C, dA, dC, lo, hi,
                                                               w.pdf_bins, 1.0, 1.0, kappa=kap)
        nvtx.range_pop()
        nvtx.range_push("covariance")
        ctx.stats_vector(mom, pdf, out=vec)
        ctx.welford_update(vec.view(1, d), wstate)
        nvtx.range_pop()
        return mom, pdf, grad

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    info = ctx.bin_info()

    stream = torch.cuda.current_stream(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ctx.profile(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.profile(False)
    prof = ctx.profile_read()
    clk = clocks.stop()
    ctx.synchronize()     # raises if a bounded device wait ran out (counts incomplete)
    ms = e0.elapsed_time(e1) / args.steps
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    # realisation split: every rank a whole map; subvolume split: one map
    value = (1 if sub else world) * n_total / (ms * 1e-3) / 1e9

    # roofline of the dominant kernel (by total time in the timed region)
    peak, peak_src = hbm_peak()
    top = max(prof.items(), key=lambda kv: kv[1][0])
    launches = sum(c for _, c in prof.values())
    fast_ms, fast_n = prof.get("k_fast", (0.0, 0))
    fast_bytes = 12.0 * n_local * args.steps            # this rank's particle reads, all launches
    bin_kernels = ["k_fast", "k_refine", "k_exact", "k_scan", "k_cursors", "k_scatter_group",
                   "k_tiles", "k_scatter_bucket", "k_hist_block"]
    bin_ms = sum(prof[k][0] for k in bin_kernels if k in prof) / args.steps
    bin_bytes = 12.0 * n_local + 4.0 * w.nshell * npix
    kap_ms = sum(prof[k][0] for k in ("k_kappa_partial", "k_adj_main", "k_moments",
                                      "k_moments_final") if k in prof)
    adj_launch = prof.get("k_adj_main", (0.0, 1))
    roof = {
        "bound": "hbm", "kernel": "k_fast",
        "achieved": fast_bytes / (fast_ms * 1e-3) / 1e9 if fast_ms else None,
        "peak": peak, "unit": "GB/s", "peak_source": f"{peak_src} hbm_gbs",
        "traffic": FAST_TRAFFIC_PER_PARTICLE * n_local / 2,
        "traffic_source": "ncu dram__bytes_read+write of a 2 x 512^3 capture, scaled per particle",
        "per_launch_bytes": 12.0 * n_local / 2, "launches": fast_n,
        "avg_launch_ms": fast_ms / max(fast_n, 1),
    }
    roof["frac"] = roof["achieved"] / peak if roof["achieved"] else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if sub else "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": w.name, "particles_per_gpu": n_local, "particles_per_map": n_total,
                   "boxes": "2000 and 6400 Mpc/h",
                   "bin_path": bin_path + (" (forced)" if args.path else " (autotuned)"),
                   "nside": w.nside, "nshell": w.nshell, "source": "Smail n(z) a=2 b=1.5 z0=0.5",
                   "l2": f"inputs larger than L2 ({12 * n_local / 1e9:.1f} GB of particles per step)",
                   "parallelism": (f"subvolumes x{world} (FP64 partial kappa and adjoint sums "
                                   "all-reduced)" if sub else f"realisations x{world}")},
        "kappa_maps_per_s": (1 if sub else world) * 1e3 / ms,
        "roofline": roof,
        "binning": {"ms": bin_ms, "algorithmic_bytes": bin_bytes,
                    "traffic": bin_bytes + BIN_SCRATCH_PER_KEY * info["keyed"],
                    "traffic_source": "algorithmic bytes + scratch bytes per keyed particle "
                                      "from an ncu capture of every binning kernel (2 x 512^3, "
                                      "Nside 1024), times this step's keyed particles",
                    "frac_of_peak": bin_bytes / (bin_ms * 1e-3) / 1e9 / peak if bin_ms else None,
                    "refined": info["refined"], "exact": info["exact"], "keyed": info["keyed"]},
        "kappa_stats_adjoint": {
            "ms": kap_ms / args.steps,
            "k_adj_main_frac_of_peak": (4.0 * w.nshell * npix + (12.0 if sub else 4.0) * npix) /
            (adj_launch[0] / adj_launch[1] * 1e-3) / 1e9 / peak if adj_launch[0] else None,
            "note": ("one pass over the counts builds the FP32 map and the adjoint sums "
                     "(counts 4 S B + map 4 B per pixel), then the moment pass" if not sub else
                     "the partial sum of the rank's counts (counts 4 S B read + 8 B written per "
                     "pixel), its all-reduce, then one pass over the counts and the summed "
                     "partials (4 S + 8 B read, map 4 B written per pixel) for the map and the "
                     "rank's adjoint sums, the moment pass, the adjoint sums' all-reduce")},
        "kernels_ms_per_step": {k: round(v[0] / args.steps, 4) for k, v in prof.items()},
        "top_kernel": top[0],
        "gpu_launches": launches,
        "clocks": clk,
    }

    # end to end: particles from pinned host memory through the C ABI each
    # step (ufc_bin_host copies them in chunks, overlapped with the binning),
    # moments and PDF back to pinned host memory
    host = None
    if not args.no_e2e:
        # pinned copies of this rank's particles; every rank must have them,
        # or no rank runs the leg (its timing takes a collective)
        err = None
        try:
            host = [torch.empty(p.shape, dtype=torch.float32, pin_memory=True) for p in parts]
        except RuntimeError as e:
            host, err = None, str(e).splitlines()[0][:160] if str(e) else type(e).__name__
        ok = torch.tensor([0 if host is None else 1], device=dev)
        if dist:
            dist.all_reduce(ok, op=dist.ReduceOp.MIN)
        if not int(ok.item()):
            host = None
            gb = sum(p.numel() * 4 for p in parts) / 1e9
            line["e2e"] = {"value": None, "unit": UNIT,
                           "unavailable": f"pinned host buffers of {gb:.1f} GB per rank could "
                                          "not be allocated" + (f": {err}" if err else
                                                                " on another rank")}
    if host is not None:
        for h_, p_ in zip(host, parts):
            h_.copy_(p_)
        out_h = torch.empty(10 + w.pdf_bins + 3, dtype=torch.float64, pin_memory=True)
        torch.cuda.synchronize()
        ke = max(2, min(args.steps, 4))

        def e2e_step():
            mom, pdf, grad = step(host)
            out_h[:10].copy_(mom, non_blocking=True)
            out_h[10:].copy_(pdf.to(torch.float64), non_blocking=True)
        e2e_step()
        torch.cuda.synchronize()
        # two windows of ke steps, the faster one reported (the host link and
        # memory are shared with other jobs; both windows are in the line)
        windows = []
        for _ in range(2):
            e0.record(stream)
            for _ in range(ke):
                e2e_step()
            e1.record(stream)
            torch.cuda.synchronize()
            windows.append(e0.elapsed_time(e1) / ke)
        ms_e = min(windows)
        if dist:
            t = torch.tensor([ms_e], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_e = float(t.item())
        h2d = int(sum(p.numel() * 4 for p in parts))
        # the host-to-device link in the same run: the same pinned buffers
        # copied into the device particle arrays (same bytes) in the
        # library's staging chunks of 2^25 particles, best of two passes
        def link_pass():
            for h_, p_ in zip(host, parts):
                for a in range(0, h_.shape[0], 1 << 25):
                    p_[a:a + (1 << 25)].copy_(h_[a:a + (1 << 25)], non_blocking=True)
        link_pass()
        torch.cuda.synchronize()
        ms_link = float("inf")
        for _ in range(2):
            e0.record(stream)
            link_pass()
            e1.record(stream)
            torch.cuda.synchronize()
            ms_link = min(ms_link, e0.elapsed_time(e1))
        link_gbs = h2d / (ms_link * 1e-3) / 1e9
        line["e2e"] = {"value": (1 if sub else world) * n_total / (ms_e * 1e-3) / 1e9, "unit": UNIT,
                       "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": int(out_h.numel() * 8 + 5 * 8 + w.nshell * 8),
                       "ms_per_step": ms_e,
                       "windows_ms_per_step": windows,
                       "h2d_link_gbs": link_gbs,
                       "h2d_link_source": "cudaMemcpyAsync of the same pinned buffers in 2^25-particle "
                                          "chunks, best of two passes, same run",
                       "frac_of_link": (h2d / (ms_e * 1e-3) / 1e9) / link_gbs}
        del host

    if not args.no_cl:
        # full-sky C_l of the step's kappa map (Sec. 3.2): a_lm, C_l
        # and band powers at lmax = 3 nside - 1
        lmax = 3 * w.nside - 1
        alm = ctx.map2alm(kap, w.nside, lmax)
        cl = ctx.alm2cl(alm, lmax)
        bp = ctx.cl_bin(cl, lmax, 10, 10, (lmax - 9) // 10)
        torch.cuda.synchronize()
        ctx.profile(True)
        e0.record(stream)
        for _ in range(3):
            ctx.map2alm(kap, w.nside, lmax, out=alm)
            ctx.alm2cl(alm, lmax, out=cl)
            ctx.cl_bin(cl, lmax, 10, 10, (lmax - 9) // 10, out=bp)
        e1.record(stream)
        torch.cuda.synchronize()
        cprof = ctx.profile_read()
        ctx.profile(False)
        ms_cl = e0.elapsed_time(e1) / 3
        npairs = 2 * w.nside
        nalm = (lmax + 1) * (lmax + 2) // 2
        # recurrence (3 multiplies, 1 subtraction) + 2 multiply-adds of the pair
        # sum per (l, m, ring pair), counted as FP64-equivalent operations
        # (the kernel evaluates them in double-float on the FP32 pipe)
        fp64 = 6.0 * npairs * nalm
        leg = cprof.get("k_legendre", (0.0, 1))
        # smoothing at the paper's 10.8 arcmin: beam, synthesis, moments, PDF
        sig = 10.8 / 60.0 * np.pi / 180.0
        work = ctx.alm_beam(alm, lmax, sig)
        sm = ctx.alm2map(work, w.nside, lmax)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(3):
            ctx.alm_beam(alm, lmax, sig, out=work)
            ctx.alm2map(work, w.nside, lmax, out=sm)
            smom, _ = ctx.map_stats(sm, w.nside, lo, hi, w.pdf_bins)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_sm = e0.elapsed_time(e1) / 3
        smh = smom.cpu().numpy()
        line["smoothed"] = {"sigma_arcmin": 10.8, "ms_per_scale": ms_sm,
                            "s2": float(smh[1]), "sigma2_s2": float(smh[7]),
                            "s2_over_sigma2_s2": float(smh[8])}
        line["cl"] = {"nside": w.nside, "lmax": lmax, "ms_per_map": ms_cl,
                      "maps_per_s": 1e3 / ms_cl,
                      "kernels_ms_per_map": {k: round(v[0] / 3, 3) for k, v in cprof.items()},
                      "k_legendre_fp64_equiv_tflops": fp64 / (leg[0] / 3 * 1e-3) / 1e12 if leg[0] else None}
        # k_legendre against the FP32 pipe: the double-float code's FP32
        # instructions per (l, m, ring pair) for l >= m + 2, as written
        # (three pair products of 7, one pair sum of 11, two multiply-adds
        # into the pair sums of 13), against 128 FP32 lanes per SM at the
        # maximum SM clock sampled during the main timed region
        if leg[0]:
            ops = 58.0 * npairs * (nalm - (2 * lmax + 1))
            nsm = torch.cuda.get_device_properties(dev).multi_processor_count
            mhz = float(clk.get("sm_max_mhz") or 2070.0) if isinstance(clk, dict) else 2070.0
            peak_alu = nsm * 128 * mhz * 1e6
            got = ops / (leg[0] / 3 * 1e-3)
            line["cl"]["roofline"] = {"bound": "alu", "kernel": "k_legendre", "achieved": got,
                                      "peak": peak_alu, "unit": "FP32 op/s", "frac": got / peak_alu,
                                      "peak_source": f"{nsm} SMs x 128 FP32 lanes x {mhz:.0f} MHz"}

    if not args.no_batched:
        line["batched_vs_serial"] = batched_leg(ctx, api, synth, dev, args.batched_real,
                                                args.batched_side)
        # small maps, where launch overheads matter: 2 x 64^3 particles, Nside 64
        line["batched_vs_serial_small"] = batched_leg(ctx, api, synth, dev, args.batched_real,
                                                      64, nside=64)

    if not args.no_snapshots:
        line["snapshots"] = snapshot_leg(ctx, api, synth, dev, w, z, chi)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        parts_h = [p[: 1 << 24].cpu().numpy() for p in parts]
        line["cpu_baseline"] = cpu_baseline(w, parts_h, counts.cpu().numpy(), A, C, (dA, dC))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
