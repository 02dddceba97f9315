"""GPU spherical-harmonic analysis (ufc_map2alm, ufc_alm2cl: the full-sky C_l
of Sec. 3.2) against the oracle's direct pixel sum, and exact properties of
the HEALPix grid at sizes beyond the oracle's reach."""
import numpy as np
import pytest

from tests.gpu_common import api_ctx

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rings(nside):
    out, start = [], 0
    for i in range(1, 4 * nside):
        n = 4 * min(i, nside, 4 * nside - i)
        out.append((start, n))
        start += n
    return out


@pytest.mark.parametrize("nside,lmax", [(4, 11), (4, 16), (8, 5), (16, 47), (32, 95), (64, 191)])
def test_alm_and_cl_match_oracle(orc, nside, lmax):
    """Random map plus a blob-like field: a_lm element by element and C_l.
    lmax above 2 nside exercises the aliasing of polar rings (m >= 4i)."""
    api, ctx = api_ctx()
    npix = 12 * nside ** 2
    rng = np.random.default_rng(nside + lmax)
    mp = (rng.normal(size=npix) + 3.0 * (rng.random(npix) < 0.01)).astype(np.float32)
    a_g = ctx.map2alm(torch.from_numpy(mp).cuda(), nside, lmax)
    cl_g = ctx.alm2cl(a_g, lmax).cpu().numpy()
    a_g = a_g.cpu().numpy()
    a_o = orc.map2alm(mp, nside, lmax)
    scale = np.abs(a_o).max()
    assert np.abs(a_g - a_o).max() <= 1e-12 * scale * lmax
    cl_o = orc.alm2cl(a_o, lmax)
    assert np.allclose(cl_g, cl_o, rtol=1e-10, atol=1e-12 * cl_o.max())


@pytest.mark.parametrize("nside", [256, 1024])
def test_grid_symmetries_large(nside):
    """Quarter turn: a_lm -> a_lm exp(-i m pi/2); mirror z -> -z:
    a_lm -> (-1)^(l+m) a_lm; constant map: a_00 = c sqrt(4 pi)."""
    api, ctx = api_ctx()
    lmax = 3 * nside - 1
    npix = 12 * nside ** 2
    rng = np.random.default_rng(nside)
    m0 = rng.normal(size=npix).astype(np.float32)
    rot = np.empty_like(m0)
    mir = np.empty_like(m0)
    rings = _rings(nside)
    for (s, n), (s2, n2) in zip(rings, rings[::-1]):
        rot[s:s + n] = np.roll(m0[s:s + n], n // 4)
        mir[s2:s2 + n2] = m0[s:s + n]
    a = ctx.map2alm(torch.from_numpy(m0).cuda(), nside, lmax)
    ar = ctx.map2alm(torch.from_numpy(rot).cuda(), nside, lmax)
    am = ctx.map2alm(torch.from_numpy(mir).cuda(), nside, lmax)
    ls = np.concatenate([np.arange(m, lmax + 1) for m in range(lmax + 1)])
    ms = np.concatenate([np.full(lmax + 1 - m, m) for m in range(lmax + 1)])
    ph = torch.from_numpy(np.exp(-0.5j * np.pi * ms)).cuda()
    sg = torch.from_numpy(((-1.0) ** (ls + ms)).astype(np.complex128)).cuda()
    scale = float(a.abs().max())
    assert float((ar - a * ph).abs().max()) <= 1e-12 * scale * lmax
    assert float((am - a * sg).abs().max()) <= 1e-12 * scale * lmax
    c = ctx.map2alm(torch.full((npix,), 1.75, dtype=torch.float32, device="cuda"), nside, lmax)
    assert float(c[0].real) == pytest.approx(1.75 * np.sqrt(4 * np.pi), rel=1e-12)


def test_band_powers_and_their_covariance(orc):
    """Binned C_l (Delta l = 10 from l = 10) of several realisations and the
    Welford covariance of the band powers, against the oracle's C_l averaged
    over the same bins and its covariance."""
    api, ctx = api_ctx()
    nside, lmax, lmin, dl, nb = 16, 47, 10, 10, 3
    rng = np.random.default_rng(21)
    d = nb
    st = api.welford_state(d)
    vs = []
    for r in range(6):
        mp = rng.normal(size=12 * nside ** 2).astype(np.float32)
        cl = ctx.alm2cl(ctx.map2alm(torch.from_numpy(mp).cuda(), nside, lmax), lmax)
        bp = ctx.cl_bin(cl, lmax, lmin, dl, nb)
        ctx.welford_update(bp.view(1, d), st)
        cl_o = orc.alm2cl(orc.map2alm(mp, nside, lmax), lmax)
        ref = cl_o[lmin:lmin + nb * dl].reshape(nb, dl).mean(axis=1)
        assert np.allclose(bp.cpu().numpy(), ref, rtol=1e-10)
        vs.append(ref)
    mean, cov, corr = ctx.welford_finalize(st, d, 1)
    _, c_o, _ = orc.covariance(np.array(vs), 1)
    assert np.allclose(cov.cpu().numpy(), c_o, rtol=1e-8, atol=1e-12 * np.abs(c_o).max())
    with pytest.raises(api.UfcError):
        ctx.cl_bin(cl, lmax, 40, 10, 1)


@pytest.mark.parametrize("nside,lmax", [(4, 11), (4, 16), (16, 47), (32, 95)])
def test_alm2map_matches_oracle(orc, nside, lmax):
    """Synthesis of random a_lm (the real field; a_l0 real) against the
    oracle's pixel-by-pixel sum; the GPU map is FP32."""
    api, ctx = api_ctx()
    rng = np.random.default_rng(100 + nside + lmax)
    n = orc.alm_size(lmax)
    a = rng.normal(size=n) + 1j * rng.normal(size=n)
    for l in range(lmax + 1):
        a[orc.alm_index(lmax, l, 0)] = a[orc.alm_index(lmax, l, 0)].real
    got = ctx.alm2map(torch.from_numpy(a).cuda(), nside, lmax).cpu().numpy()
    ref = orc.alm2map(a, nside, lmax)
    assert np.abs(got - ref).max() <= 2e-6 * np.abs(ref).max()


def test_smoothing_chain_matches_oracle(orc):
    """Map -> a_lm -> Gaussian beam (r.m.s. radius 2 pixels) -> map -> moments
    and PDF, against the oracle's chain; moments at 1e-9 on the GPU's map."""
    api, ctx = api_ctx()
    nside, lmax = 32, 95
    rng = np.random.default_rng(77)
    mp = (rng.normal(size=12 * nside ** 2) + 5.0 * (rng.random(12 * nside ** 2) < 0.01)).astype(np.float32)
    sigma = 2 * np.sqrt(4 * np.pi / (12 * nside ** 2))
    a = ctx.map2alm(torch.from_numpy(mp).cuda(), nside, lmax)
    sm = ctx.alm2map(ctx.alm_beam(a, lmax, sigma), nside, lmax)
    a_o = orc.map2alm(mp, nside, lmax) * np.repeat(
        [orc.gauss_beam(sigma, lmax)], 1, axis=0)[0][[l for m in range(lmax + 1) for l in range(m, lmax + 1)]]
    ref = orc.alm2map(a_o, nside, lmax)
    smh = sm.cpu().numpy()
    assert np.abs(smh - ref).max() <= 2e-6 * np.abs(ref).max()
    lo, hi = float(smh.min()), float(smh.max()) * 0.9
    mom, pdf = ctx.map_stats(sm, nside, lo, hi, 50)
    m_or = orc.moments(smh)
    mg = mom.cpu().numpy()
    for i in (1, 2, 3, 4, 5, 6, 7, 8):
        assert mg[i] == pytest.approx(m_or[i], rel=1e-9), i
    assert np.array_equal(pdf.cpu().numpy(), orc.pdf(smh, lo, hi, 50))


def test_map_stats_equals_kappa_stats(orc):
    """ufc_map_stats on the kappa map gives ufc_kappa_stats's moments and PDF
    bit for bit (same per-block sums, same second pass)."""
    api, ctx = api_ctx()
    nside, S = 64, 8
    rng = np.random.default_rng(3)
    counts = torch.from_numpy(rng.poisson(4.0, size=(S, 12 * nside ** 2)).astype(np.int32)).cuda()
    A = rng.uniform(0.001, 0.01, size=S)
    kap, mom, pdf = ctx.kappa_stats(counts, A, 0.1, -0.1, 0.4, 40)
    mom2, pdf2 = ctx.map_stats(kap, nside, -0.1, 0.4, 40)
    assert torch.equal(mom, mom2) and torch.equal(pdf, pdf2)
