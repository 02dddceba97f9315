"""GPU parity of the kappa map (Eq. 6), moments (Eq. 12-13), PDF (Sec. 3.3),
adjoint gradients and the Welford covariance (Eq. 10-11)."""
import numpy as np
import pytest

from paper_1801_05745_gb300 import synth
from tests.gpu_common import api_ctx, both_boxes, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _map(orc, api, ctx, nside, nshell, n, seed, kind=1):
    x1 = synth.particles_numpy(n, 2000.0, 5.0, seed)
    x2 = synth.particles_numpy(n, 6400.0, 20.0, seed + 1)
    z = np.linspace(0.1, 1.5, nshell + 1)
    chi = orc.chi_edges(0.3, 0.7, 1, z)
    split = int(np.argmin(np.abs(chi - 1000.0)))
    b1a, b1o = both_boxes(api, orc, 2000.0, [1000.0] * 3, n, 0, split)
    b2a, b2o = both_boxes(api, orc, 6400.0, [3200.0] * 3, n, split, nshell)
    counts = ctx.bin([to_dev(x1), to_dev(x2)], [b1a, b2a], chi, nside)
    kw = dict(kind=kind, z_s=1.5, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5)
    return counts, z, (b1a, b2a), (b1o, b2o), kw


def kappa_gate(k_gpu, k_or, A, counts):
    """|dk| <= 1e-5 max(|k|, sum_b |A_b| n_bp + |C|) (scale of the cancelling terms)."""
    scale = (np.abs(A)[:, None] * counts).sum(0)
    return np.abs(k_gpu.astype(np.float64) - k_or.astype(np.float64)) <= 1e-5 * np.maximum(
        np.abs(k_or), scale) + 1e-30


@pytest.mark.parametrize("nside,nshell,kind", [(16, 8, 0), (64, 20, 1), (256, 40, 1)])
def test_kappa_moments_pdf(orc, nside, nshell, kind):
    api, ctx = api_ctx()
    counts, z, ba, bo, kw = _map(orc, api, ctx, nside, nshell, 400_000, 1234 + nside, kind)
    A, B, C = orc.kappa_coeffs(0.3, 0.7, 1, list(bo), z, nside, orc.make_source(**kw))
    k_or = orc.kappa_map(counts.cpu().numpy(), A, C)
    lo, hi = float(k_or.min()) * 0.9, float(k_or.max()) * 0.8
    kap, mom, pdf = ctx.kappa_stats(counts, A, C, lo, hi, 200)
    kg = kap.cpu().numpy()
    cn = counts.cpu().numpy()
    assert kappa_gate(kg, k_or, A, cn).all()
    assert (kg == k_or).mean() > 0.999     # nearly always the same rounding
    # moments and PDF on the GPU's own kappa
    m_or = orc.moments(kg)
    mg = mom.cpu().numpy()
    for i in range(10):
        assert mg[i] == pytest.approx(m_or[i], rel=1e-9, abs=1e-15 * abs(m_or[1]) ** 0.5 * (i == 0)), i
    assert np.array_equal(pdf.cpu().numpy(), orc.pdf(kg, lo, hi, 200))


def test_pdf_values_on_bin_edges(orc):
    """kappa = n 2^-12 lands exactly on the edges of 96 bins over
    [0, 96 2^-12): the half-open rule and the exact FP64 fallback decide."""
    api, ctx = api_ctx()
    npix = 12 * 16 * 16
    counts = torch.from_numpy((np.arange(npix, dtype=np.int32) % 98).reshape(1, npix)).cuda()
    A = np.array([2.0 ** -12])
    lo, hi, nb = 0.0, 96 * 2.0 ** -12, 96
    kap, mom, pdf = ctx.kappa_stats(counts, A, 0.0, lo, hi, nb)
    kg = kap.cpu().numpy()
    assert np.array_equal(kg, (np.arange(npix) % 98) * np.float32(2.0 ** -12))
    p = pdf.cpu().numpy()
    assert np.array_equal(p, orc.pdf(kg, lo, hi, nb))
    assert p[nb + 1] > 0 and p[:nb].min() > 0     # values at hi overflow
    # a range with an offset lo and a non-power-of-two width
    kap2, _, pdf2 = ctx.kappa_stats(counts, A, 0.0, 0.001, 0.0191, 37)
    assert np.array_equal(pdf2.cpu().numpy(), orc.pdf(kap2.cpu().numpy(), 0.001, 0.0191, 37))


@pytest.mark.parametrize("kind,units", [(0, 1), (1, 1), (1, 0)])
def test_backward_vs_complex_step(orc, kind, units):
    api, ctx = api_ctx()
    nside, nshell = 32, 12
    counts, z, ba, bo, kw = _map(orc, api, ctx, nside, nshell, 300_000, 99 + kind, kind)
    kw["z_s"] = 1.5
    cosmo = api.make_cosmo(0.3, 0.7, units)
    A, B, C, dA, dC = api.kappa_coeffs(cosmo, list(ba), z, nside, api.make_source(**kw), derivs=True)
    rng = np.random.default_rng(5)
    g = rng.normal(size=counts.shape[1]).astype(np.float32)
    cn = counts.cpu().numpy()
    G_or = orc.kappa_stat_grads(cn, nside, 0.3, 0.7, units, list(bo), z, orc.make_source(**kw), g)
    for wv, ws, use_g in [(1.0, 0.0, False), (0.0, 1.0, False), (0.0, 0.0, True), (0.7, -0.3, True)]:
        grad, Gb, H = ctx.kappa_backward(counts, A, C, dA, dC, wv, ws, to_dev(g) if use_g else None)
        ref = wv * G_or[0] + ws * G_or[1] + (G_or[2] if use_g else 0.0)
        scale = np.abs(wv * G_or[0]).max() + np.abs(ws * G_or[1]).max() + (np.abs(G_or[2]).max() if use_g else 0)
        assert np.allclose(grad, ref, rtol=1e-9, atol=1e-9 * scale), (wv, ws, use_g, grad, ref)


def test_welford_vs_oracle_covariance(orc):
    api, ctx = api_ctx()
    rng = np.random.default_rng(3)
    v = rng.normal(size=(150, 33)) @ rng.normal(size=(33, 33)) + 5.0
    d = v.shape[1]
    st = api.welford_state(d)
    vt = torch.from_numpy(v).cuda()
    ctx.welford_update(vt[:70], st)
    # a second state merged in (the realisation-sharded path)
    st2 = api.welford_state(d)
    ctx.welford_update(vt[70:], st2)
    ctx.welford_merge(st, st2, d)
    for ddof in (0, 1):
        mean, cov, corr = ctx.welford_finalize(st, d, ddof)
        m_o, c_o, r_o = orc.covariance(v, ddof)
        assert np.allclose(mean.cpu().numpy(), m_o, rtol=1e-12, atol=1e-12)
        assert np.allclose(cov.cpu().numpy(), c_o, rtol=1e-9, atol=1e-12)
        assert np.allclose(corr.cpu().numpy(), r_o, rtol=1e-9, atol=1e-12)


def test_welford_many_vectors_equal_one_at_a_time():
    """One update over 64 vectors (the batched call's form) gives the state of
    64 single-vector updates; repeated, so that a thread that reads the count
    before another one advanced it (a race within the update) would show."""
    api, ctx = api_ctx()
    rng = np.random.default_rng(64)
    d = 206
    for rep in range(6):
        v = rng.normal(size=(64, d)) * rng.uniform(0.1, 10.0, size=d) + rng.normal(size=d)
        vt = torch.from_numpy(v).cuda()
        st_many = api.welford_state(d)
        st_one = api.welford_state(d)
        ctx.welford_update(vt, st_many)
        for r in range(64):
            ctx.welford_update(vt[r:r + 1], st_one)
        torch.cuda.synchronize()
        assert st_many[0].item() == 64.0
        assert torch.allclose(st_many, st_one, rtol=1e-12, atol=1e-12 * float(st_one.abs().max()))


def test_welford_host_calls_match_device_calls():
    """ufc_welford_update_host / ufc_welford_merge_host (the multi-process
    path's host states) against the device update and merge."""
    api, ctx = api_ctx()
    rng = np.random.default_rng(7)
    d = 46
    v = rng.normal(size=(40, d)) * 3.0 + 1.0
    sd, sd2 = api.welford_state(d), api.welford_state(d)
    ctx.welford_update(torch.from_numpy(v[:25]).cuda(), sd)
    ctx.welford_update(torch.from_numpy(v[25:]).cuda(), sd2)
    ctx.welford_merge(sd, sd2, d)
    sh, sh2 = np.zeros(1 + d + d * d), np.zeros(1 + d + d * d)
    api.welford_update_host(v[:25], sh)
    api.welford_update_host(v[25:], sh2)
    api.welford_merge_host(sh, sh2, d)
    torch.cuda.synchronize()
    assert np.allclose(sd.cpu().numpy(), sh, rtol=1e-12, atol=1e-12 * np.abs(sh).max())


def test_welford_at_the_largest_statistics_vector(orc):
    """d = 6 + 4096 PDF bins: the update's shared memory (2 d doubles) is
    above the 48 KB default and must still launch; covariance against the
    oracle on a few rows and columns."""
    api, ctx = api_ctx()
    rng = np.random.default_rng(4102)
    d, R = 6 + 4096, 12
    v = rng.normal(size=(R, d)) + 3.0
    st = api.welford_state(d)
    ctx.welford_update(torch.from_numpy(v).cuda(), st)
    mean, cov, corr = ctx.welford_finalize(st, d, 1)
    torch.cuda.synchronize()
    cols = np.array([0, 1, 5, 6, 777, 4101])
    m_o, c_o, _ = orc.covariance(v[:, cols], 1)
    assert np.allclose(mean.cpu().numpy()[cols], m_o, rtol=1e-12, atol=1e-12)
    assert np.allclose(cov.cpu().numpy()[np.ix_(cols, cols)], c_o, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("nside,nshell", [(64, 20), (256, 40)])
def test_delta_map_stats_and_gradient(orc, nside, nshell):
    """Overdensity map of Eq. 7 through ufc_kappa_stats with the library's
    delta coefficients: map against the oracle's definition, moments and
    PDF on the GPU's map, and d var / d(Omega_m, h) from ufc_kappa_backward
    against 4th-order central differences of the FP64 map (Mpc units, where
    both parameters enter through chi)."""
    api, ctx = api_ctx()
    counts, z, ba, bo, kw = _map(orc, api, ctx, nside, nshell, 400_000, 777 + nside)
    cosmo = api.make_cosmo(0.3, 0.7, 0)
    A, C, dA, dC = api.delta_coeffs(cosmo, list(ba), z, nside, derivs=True)
    Ao, Co = orc.delta_coeffs(0.3, 0.7, 0, list(bo), z, nside)
    assert np.allclose(A, Ao, rtol=1e-12) and C == Co == 1.0
    cn = counts.cpu().numpy()
    d_or = orc.kappa_map(cn, Ao, Co)
    lo, hi = -1.0, float(d_or.max()) * 0.5
    dmap, mom, pdf = ctx.kappa_stats(counts, A, C, lo, hi, 100)
    dg = dmap.cpu().numpy()
    assert kappa_gate(dg, d_or, Ao, cn).all()
    m_or = orc.moments(dg)
    mg = mom.cpu().numpy()
    for i in (1, 2, 3, 4, 5):
        assert mg[i] == pytest.approx(m_or[i], rel=1e-9), i
    assert np.array_equal(pdf.cpu().numpy(), orc.pdf(dg, lo, hi, 100))
    grad, _, _ = ctx.kappa_backward(counts, A, C, dA, dC, 1.0, 0.0)

    def var(om, h):
        a, c = orc.delta_coeffs(om, h, 0, list(bo), z, nside)
        d = a @ cn.astype(np.float64) - c
        return float(np.mean((d - d.mean()) ** 2))
    for j, (om, h) in enumerate([(1, 0), (0, 1)]):
        e = 1e-4
        f = lambda t: var(0.3 + om * t, 0.7 + h * t)
        fd = (-f(2 * e) + 8 * f(e) - 8 * f(-e) + f(-2 * e)) / (12 * e)
        assert grad[j] == pytest.approx(fd, rel=1e-6), j


def test_backward_large_counts_flush_path(orc):
    """Counts near 2^31 in some pixels push the adjoint's bound on its 64-bit
    lane sums past 2^61 within a launch, so the sums are flushed into the
    128-bit rows mid-launch; the gradient must still match the oracle's
    complex step.  A 20 Mpc/h box keeps |kappa| near 4000, below the 2^14
    fixed-point range."""
    api, ctx = api_ctx()
    nside, nshell = 512, 6
    npix = 12 * nside ** 2
    z = np.linspace(0.1, 1.0, nshell + 1)
    rng = np.random.default_rng(11)
    cn = rng.poisson(3.0, size=(nshell, npix)).astype(np.int32)
    big = rng.choice(npix, size=4096, replace=False)
    cn[:, big] = (2 ** 31 - 1 - rng.integers(0, 1000, size=(nshell, big.size))).astype(np.int32)
    kw = dict(kind=0, z_s=1.5)
    n_total = 500_000
    cosmo = api.make_cosmo(0.3, 0.7, 1)
    ba = [api.make_box(20.0, [10.0] * 3, n_total, 0, nshell)]
    bo = [orc.make_box(20.0, [10.0] * 3, n_total, 0, nshell)]
    A, B, C, dA, dC = api.kappa_coeffs(cosmo, ba, z, nside, api.make_source(**kw), derivs=True)
    kmax = float((A[:, None] * cn[:, big].astype(np.float64)).sum(0).max())
    assert 100.0 < kmax < 8000.0
    grad, _, _ = ctx.kappa_backward(torch.from_numpy(cn).cuda(), A, C, dA, dC, 1.0, 0.5)
    G_or = orc.kappa_stat_grads(cn, nside, 0.3, 0.7, 1, bo, z, orc.make_source(**kw))
    ref = G_or[0] + 0.5 * G_or[1]
    scale = np.abs(G_or[0]).max() + 0.5 * np.abs(G_or[1]).max()
    assert np.allclose(grad, ref, rtol=1e-8, atol=1e-9 * scale), (grad, ref)


@pytest.mark.parametrize("nside,nshell,use_g", [(64, 20, False), (128, 60, True), (64, 80, False)])
def test_fused_map_and_adjoint_equal_separate_calls(orc, nside, nshell, use_g):
    """ufc_kappa_stats_backward (one read of the counts) against
    ufc_kappa_stats then ufc_kappa_backward: the FP32 map, the PDF and the
    gradient with G_b and H bit for bit; the moments to the last bits (the
    mean's partial sums run over another grid) and against the oracle on
    the map.  80 shells take two launch windows of the adjoint."""
    api, ctx = api_ctx()
    counts, z, ba, bo, kw = _map(orc, api, ctx, nside, nshell, 300_000, 99 + nshell)
    A, B, C, dA, dC = api.kappa_coeffs(api.make_cosmo(), list(ba), z, nside,
                                       api.make_source(**kw), derivs=True)
    npix = 12 * nside * nside
    g = torch.linspace(-1.0, 1.0, npix, device="cuda") if use_g else None
    lo, hi = -0.02, 0.1
    kap, mom, pdf = ctx.kappa_stats(counts, A, C, lo, hi, 64)
    grad, G, H = ctx.kappa_backward(counts, A, C, dA, dC, 0.7, 1.3, g)
    kf, mf, pf, gf, Gf, Hf = ctx.kappa_stats_backward(counts, A, C, dA, dC, lo, hi, 64, 0.7, 1.3, g)
    torch.cuda.synchronize()
    assert torch.equal(kf, kap)
    assert torch.equal(pf, pdf)
    assert np.array_equal(gf, grad) and np.array_equal(Gf, G) and Hf == H
    mo = orc.moments(kf.cpu().numpy())
    assert np.allclose(mf.cpu().numpy(), mom.cpu().numpy(), rtol=1e-13, atol=1e-18)
    assert np.allclose(mf.cpu().numpy(), mo, rtol=1e-9, atol=1e-15)
