"""GPU parity of the subvolume combination (Sec. 2.4): the particles of each
box are split into contiguous shards binned separately (virtual ranks on one
GPU), the shards' FP64 partial kappa sums are added (the all-reduce), and the
map, its moments and PDF and the adjoint gradient built from the summed
partials and the shards' own counts are compared with the single-pass calls
on the whole counts and with the oracle."""
import numpy as np
import pytest

from paper_1801_05745_gb300 import parallel, synth
from tests.gpu_common import api_ctx, both_boxes, to_dev
from tests.test_gpu_stats import kappa_gate

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _shards(orc, api, ctx, nside, nshell, n, seed, nsub):
    x1 = synth.particles_numpy(n, 2000.0, 5.0, seed)
    x2 = synth.particles_numpy(n, 6400.0, 20.0, seed + 1)
    z = np.linspace(0.1, 1.5, nshell + 1)
    chi = orc.chi_edges(0.3, 0.7, 1, z)
    split = int(np.argmin(np.abs(chi - 1000.0)))
    b1a, b1o = both_boxes(api, orc, 2000.0, [1000.0] * 3, n, 0, split)
    b2a, b2o = both_boxes(api, orc, 6400.0, [3200.0] * 3, n, split, nshell)
    full = ctx.bin([to_dev(x1), to_dev(x2)], [b1a, b2a], chi, nside)
    parts = []
    for r in range(nsub):
        a, b = parallel.shard_range(n, r, nsub, align=4)
        parts.append(ctx.bin([to_dev(x1[a:b]), to_dev(x2[a:b])], [b1a, b2a], chi, nside))
    kw = dict(kind=1, z_s=1.5, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5)
    return full, parts, z, (b1a, b2a), (b1o, b2o), kw


@pytest.mark.parametrize("nside,nshell,nsub", [(64, 20, 2), (128, 60, 3), (32, 100, 2)])
def test_partial_sums_map_and_gradient(orc, nside, nshell, nsub):
    """100 shells take two launch windows of the adjoint."""
    api, ctx = api_ctx()
    full, parts, z, ba, bo, kw = _shards(orc, api, ctx, nside, nshell, 300_000, 7 + nshell, nsub)
    torch.cuda.synchronize()
    assert torch.equal(sum(p.to(torch.int64) for p in parts), full.to(torch.int64))
    A, B, C, dA, dC = api.kappa_coeffs(api.make_cosmo(), list(ba), z, nside,
                                       api.make_source(**kw), derivs=True)
    npix = 12 * nside * nside
    cn = full.cpu().numpy()
    # the partials add up to sum_b A_b n_bp of the whole counts (FP64)
    E = sum(ctx.kappa_partial(p, A) for p in parts)
    ref = A @ cn.astype(np.float64)
    scale = np.abs(A) @ cn.astype(np.float64)
    assert np.all(np.abs(E.cpu().numpy() - ref) <= 1e-12 * scale + 1e-300)
    # the map from the summed partials against the single pass and the oracle
    lo, hi = -0.02, 0.1
    ks, ms, ps = ctx.kappa_stats_partial(E, C, lo, hi, 64)
    k1, m1, p1 = ctx.kappa_stats(full, A, C, lo, hi, 64)
    ksn, k1n = ks.cpu().numpy(), k1.cpu().numpy()
    # both round values known to ~2^-48 of the cancelling terms: one FP32
    # unit apart at most, more only where kappa itself is far below them
    ulp = np.spacing(np.abs(k1n).astype(np.float32)).astype(np.float64)
    diff = np.abs(ksn.astype(np.float64) - k1n.astype(np.float64))
    assert np.all(diff <= np.maximum(ulp, 1e-12 * (scale + abs(C))))
    assert (diff > 0).sum() <= max(5, npix // 10_000)
    assert kappa_gate(ksn, orc.kappa_map(cn, A, C), A, cn).all()
    assert np.allclose(ms.cpu().numpy(), m1.cpu().numpy(), rtol=1e-12, atol=1e-18)
    assert np.allclose(ms.cpu().numpy(), orc.moments(ksn), rtol=1e-9, atol=1e-15)
    assert np.array_equal(ps.cpu().numpy(), orc.pdf(ksn, lo, hi, 64))
    # the adjoint: each shard's share against the summed partials, the
    # per-shell sums added, the chain rule on the host
    g = torch.linspace(-1.0, 1.0, npix, device="cuda")
    shares = []
    for i, p in enumerate(parts):
        sm, kf, mf, pf = ctx.kappa_adjoint_sums(p, E, C, g, lo, hi, 64, want_map=(i == 0))
        if i == 0:        # the same read of the counts gives the same map
            assert torch.equal(kf, ks) and torch.equal(pf, ps)
            # moments to the last bits (the mean's partial sums over another grid)
            assert np.allclose(mf.cpu().numpy(), ms.cpu().numpy(), rtol=1e-13, atol=1e-18)
        shares.append(sm)
    S = nshell
    for sm in shares[1:]:     # whole-map power sums: the same in every shard
        assert np.array_equal(sm[4 * S:], shares[0][4 * S:])
    tot = np.concatenate([sum(sm[:4 * S] for sm in shares), shares[0][4 * S:]])
    assert np.array_equal(tot[3:4 * S:4], cn.sum(1).astype(np.float64))    # N_b
    grad, G, H = api.kappa_grad_from_sums(tot, S, nside, dA, dC, 0.7, 1.3)
    grad1, G1, H1 = ctx.kappa_backward(full, A, C, dA, dC, 0.7, 1.3, g)
    assert np.allclose(grad, grad1, rtol=1e-10, atol=1e-12 * np.abs(grad1).max())
    assert np.allclose(G, G1, rtol=1e-10, atol=1e-12 * np.abs(G1).max())
    assert H == pytest.approx(H1, rel=1e-12)
    # and against the oracle's complex step on the whole counts
    G_or = orc.kappa_stat_grads(cn, nside, 0.3, 0.7, 1, list(bo), z, orc.make_source(**kw),
                                g.cpu().numpy())
    want = 0.7 * G_or[0] + 1.3 * G_or[1] + G_or[2]
    sc = 0.7 * np.abs(G_or[0]).max() + 1.3 * np.abs(G_or[1]).max() + np.abs(G_or[2]).max()
    assert np.allclose(grad, want, rtol=1e-9, atol=1e-9 * sc), (grad, want)


def test_subvolume_kappa_one_process_equals_calls(orc):
    """parallel.subvolume_kappa without a process group (one subvolume) is
    the sequence of library calls; with a single shard its map equals the
    single-pass map up to rare last-unit differences."""
    api, ctx = api_ctx()
    full, parts, z, ba, bo, kw = _shards(orc, api, ctx, 64, 20, 200_000, 31, 1)
    A, B, C, dA, dC = api.kappa_coeffs(api.make_cosmo(), list(ba), z, 64, api.make_source(**kw),
                                       derivs=True)
    k, m, p, grad, G, H = parallel.subvolume_kappa(ctx, full, A, C, -0.02, 0.1, 50, dA=dA, dC=dC,
                                                   w_var=1.0, w_skew=1.0)
    k2, m2, p2 = parallel.subvolume_kappa(ctx, full, A, C, -0.02, 0.1, 50)
    assert torch.equal(k, k2) and torch.equal(p, p2)
    g1, _, _ = ctx.kappa_backward(full, A, C, dA, dC, 1.0, 1.0)
    assert np.allclose(grad, g1, rtol=1e-10, atol=1e-12 * np.abs(g1).max())


def test_partial_calls_reject_bad_arguments():
    api, ctx = api_ctx()
    npix = 12 * 16 * 16
    counts = torch.zeros((4, npix), dtype=torch.int32, device="cuda")
    A = np.ones(4)
    buf = torch.zeros(npix + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(api.UfcError):
        ctx.kappa_partial(counts, A, out=buf[1:])          # 8-byte, not 16-byte aligned
    with pytest.raises(api.UfcError):
        ctx.kappa_stats_partial(buf[1:], 0.0, -1.0, 1.0, 10)
    E = ctx.kappa_partial(counts, A)
    with pytest.raises(api.UfcError):
        ctx.kappa_stats_partial(E, float("nan"), -1.0, 1.0, 10)
    with pytest.raises(api.UfcError):
        ctx.kappa_stats_partial(E, 0.0, 1.0, -1.0, 10)     # empty PDF range
    with pytest.raises(api.UfcError):
        api.kappa_grad_from_sums(np.full(4 * 4 + 4, np.nan), 4, 16, np.ones(20), np.ones(5))
