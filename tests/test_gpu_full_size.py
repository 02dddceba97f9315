"""Parity at the benchmarked size: the full map of the benchmark (two nested
boxes of 1024^3 particles, 60 shells z = 0.1 - 1.5, Nside 1024, Smail n(z)),
generated exactly as bench.py generates it, binned by the library and by the
oracle's OpenMP binning on the same bytes.

Paths that only occur at this size are covered here: dense-key chunks of
about 10^9 keys, both scatter passes over 4 GB of keys, the refine queue at
the real density of undecided particles, the moment pass over 12.6M pixels
and the adjoint over 60 shells at Nside 1024 (Eq. 5, 6, 8, 12; Sec. 2.4)."""
import os

import numpy as np
import pytest

from tests.gpu_common import api_ctx

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _host_ram_bytes():
    try:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    except (ValueError, OSError):
        return 0


def test_full_size_map_against_oracle(orc):
    import bench
    from paper_1801_05745_gb300 import synth, workloads

    api, ctx = api_ctx()
    if torch.cuda.mem_get_info()[0] < (80 << 30) or _host_ram_bytes() < (64 << 30):
        pytest.skip("needs 80 GB of free device memory and 64 GB of host memory")
    w = workloads.full()
    z, chi, split = bench.shells(w, api=api)
    S, nside = w.nshell, w.nside
    npix = 12 * nside * nside
    boxes_a = [api.make_box(2000.0, [1000.0] * 3, w.boxes[0].n, 0, split),
               api.make_box(6400.0, [3200.0] * 3, w.boxes[1].n, split, S)]
    boxes_o = [orc.make_box(2000.0, [1000.0] * 3, w.boxes[0].n, 0, split),
               orc.make_box(6400.0, [3200.0] * 3, w.boxes[1].n, split, S)]
    parts = [synth.particles_torch(b.n, b.L, b.sigma, synth.seed_for(3, 0, k), device="cuda")
             for k, b in enumerate(w.boxes)]
    counts = ctx.bin(parts, boxes_a, chi, nside)
    info = ctx.bin_info()
    assert info["refined"] > 0 and info["keyed"] > 9e8   # the real density of undecided images

    # ---- counts: bit for bit against the oracle on the same bytes (Eq. 5, 8)
    ref = np.zeros((S, npix), dtype=np.int32)
    for k in range(2):
        x = parts[k].cpu().numpy()
        _, inv, _ = orc.bin_counts_omp(x, boxes_o[k], chi, nside, ref)
        assert inv == 0
        del x
    del parts
    got = counts.cpu().numpy()
    ndiff = int(np.count_nonzero(got != ref))
    assert ndiff == 0, f"{ndiff} (shell, pixel) cells differ from the oracle"
    assert int(ref.sum()) == info["keyed"]
    del got

    # ---- kappa map (Eq. 6) against the oracle's map of its own counts
    src = dict(kind=1, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5)
    A, B, C, dA, dC = api.kappa_coeffs(api.make_cosmo(w.omega_m, w.h, 1), boxes_a, z, nside,
                                       api.make_source(**src), derivs=True)
    Ao, Bo, Co = orc.kappa_coeffs(w.omega_m, w.h, 1, boxes_o, z, nside, orc.make_source(**src))
    k_or = orc.kappa_map(ref, Ao, Co)
    scale = np.zeros(npix)
    k64 = np.full(npix, -Co)
    for b in range(S):              # shell by shell: no [S, npix] FP64 temporary
        cb = ref[b].astype(np.float64)
        scale += abs(Ao[b]) * cb
        k64 += Ao[b] * cb
    lo = float(k64.mean() - 6 * k64.std())
    hi = float(k64.mean() + 6 * k64.std())
    kap, mom, pdf = ctx.kappa_stats(counts, A, C, lo, hi, w.pdf_bins)
    kg = kap.cpu().numpy()
    bad = np.abs(kg.astype(np.float64) - k_or) > 1e-5 * np.maximum(np.abs(k_or), scale + abs(Co))
    assert not bad.any(), f"{int(bad.sum())} kappa pixels outside the 1e-5 gate"

    # ---- moments (Eq. 12-13) and PDF on the GPU's FP32 map
    m_or = orc.moments(kg)
    assert np.allclose(mom.cpu().numpy(), m_or, rtol=1e-9, atol=0)
    assert np.array_equal(pdf.cpu().numpy(), orc.pdf(kg, lo, hi, w.pdf_bins))

    # ---- adjoint of var + skew of the unrounded map, counts fixed: G_b and
    # H against their definitions G_b = sum_p gbar_p n_bp, H = sum_p gbar_p
    # with gbar = d(var + skew)/d kappa evaluated in FP64 on the host
    grad, G, H = ctx.kappa_backward(counts, A, C, dA, dC, 1.0, 1.0)
    d = k64 - k64.mean()
    mu2 = float(np.mean(d * d))
    mu3 = float(np.mean(d * d * d))
    N = float(npix)
    gbar = 2.0 * d / N + 3.0 / N * (d * d - mu2) * mu2 ** -1.5 - 3.0 * mu3 * mu2 ** -2.5 * d / N
    G_np = np.empty(S)
    G_scale = np.empty(S)
    ag = np.abs(gbar)
    for b in range(S):
        cb = ref[b].astype(np.float64)
        G_np[b] = float(np.dot(cb, gbar))
        G_scale[b] = float(np.dot(cb, ag))
    H_np = float(gbar.sum())
    assert np.all(np.abs(G - G_np) <= 1e-9 * G_scale + 1e-12 * G_scale.max()), (G, G_np)
    assert abs(H - H_np) <= 1e-9 * float(ag.sum())
    grad_np = dA @ G_np - dC * H_np
    g_scale = np.abs(dA) @ G_scale + np.abs(dC) * float(ag.sum())
    assert np.all(np.abs(grad - grad_np) <= 1e-9 * g_scale), (grad, grad_np)
    assert grad[1] == 0.0                  # h cancels for lengths in Mpc/h
    ctx.synchronize()
