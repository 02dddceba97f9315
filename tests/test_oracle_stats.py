"""Pins of the oracle's kappa map (Eq. 6), moments (Eq. 12-13), PDF and
covariance (Eq. 10-11): hand-computed values, textbook identities, numpy's
covariance, and complex-step against finite differences."""
import numpy as np
import pytest


def test_moments_hand_computed(orc):
    # {-1, 0, 1, 2}: mean 1/2; deviations -3/2,-1/2,1/2,3/2
    m = orc.moments(np.array([-1, 0, 1, 2], np.float32))
    assert m[0] == 0.5
    assert m[1] == pytest.approx(1.25, abs=0)
    assert m[2] == pytest.approx(0.0, abs=1e-15)
    assert m[3] == pytest.approx((2 * 1.5 ** 4 + 2 * 0.5 ** 4) / 4, abs=0)
    assert m[5] == pytest.approx(2.5625 / 1.25 ** 2 - 3)
    N = 4.0
    assert m[6] == pytest.approx((N - 1) * 1.25 / N)
    assert m[7] == pytest.approx((N - 1) ** 2 / N ** 3 * 2.5625 - (N - 1) * (N - 3) / N ** 3 * 1.25 ** 2)
    assert m[9] == 4.0


def test_moments_skewed_and_invariances(orc):
    # {0, 0, 0, 4}: mean 1, mu2 = 3, mu3 = (3*(-1)^3 + 27)/4 = 6, skew = 6/3^1.5
    m = orc.moments(np.array([0, 0, 0, 4], np.float32))
    assert m[1] == 3.0 and m[2] == 6.0 and m[4] == pytest.approx(6 / 3 ** 1.5, rel=1e-15)
    rng = np.random.default_rng(0)
    x = rng.gamma(2.0, size=100_000).astype(np.float32)
    a = orc.moments(x)
    b = orc.moments((x * np.float32(2.0)))          # exact scaling by 2
    assert b[1] == pytest.approx(4 * a[1], rel=1e-14)
    assert b[3] == pytest.approx(16 * a[3], rel=1e-14)
    assert b[4] == pytest.approx(a[4], rel=1e-13)
    # against numpy's moments of the promoted data (two-pass, library)
    xd = x.astype(np.float64)
    d = xd - xd.mean()
    assert a[1] == pytest.approx((d ** 2).mean(), rel=1e-12)
    assert a[2] == pytest.approx((d ** 3).mean(), rel=1e-11)
    assert a[3] == pytest.approx((d ** 4).mean(), rel=1e-12)
    # Eq. 13 tends to (mu4 - mu2^2)/N for large N
    assert a[7] == pytest.approx((a[3] - a[1] ** 2) / len(x), rel=1e-4)


def test_pdf_hand_example(orc):
    k = np.array([-1.0, 0.0, 0.1, 0.25, 0.5, 0.999, 1.0, 2.0, np.nan], np.float32)
    p = orc.pdf(k, 0.0, 1.0, 4)
    # bins [0,.25) [.25,.5) [.5,.75) [.75,1), under, over, nan
    assert list(p) == [2, 1, 1, 1, 1, 2, 1]


def test_covariance_against_numpy(orc):
    rng = np.random.default_rng(1)
    v = rng.normal(size=(150, 12)) @ rng.normal(size=(12, 12))
    for ddof in (0, 1):
        mean, cov, corr = orc.covariance(v, ddof)
        assert np.allclose(mean, v.mean(0), rtol=1e-13, atol=1e-14)
        assert np.allclose(cov, np.cov(v, rowvar=False, ddof=ddof), rtol=1e-12, atol=1e-13)
        assert np.allclose(corr, np.corrcoef(v, rowvar=False), rtol=1e-12, atol=1e-13)


def _small_map(orc, nside=8, nshell=4, seed=3):
    rng = np.random.default_rng(seed)
    npix = 12 * nside * nside
    counts = rng.poisson(3.0, size=(nshell, npix)).astype(np.int32)
    z = np.linspace(0.2, 1.0, nshell + 1)
    boxes = [orc.make_box(2000.0, [1000.0] * 3, 64 ** 3, 0, nshell)]
    return counts, z, boxes


def test_single_particle_moves_one_pixel(orc):
    counts, z, boxes = _small_map(orc)
    src = orc.make_source(kind=0, z_s=1.2)
    A, B, C = orc.kappa_coeffs(0.3, 0.7, 1, boxes, z, 8, src)
    zero = np.zeros_like(counts)
    one = zero.copy()
    one[2, 77] = 1
    k0 = orc.kappa_map(zero, A, C)
    k1 = orc.kappa_map(one, A, C)
    assert np.all(k0 == np.float32(-C))
    diff = np.nonzero(k1 != k0)[0]
    assert list(diff) == [77] and k1[77] == np.float32(A[2] - C)


def test_mean_identity_and_zero_matter(orc):
    counts, z, boxes = _small_map(orc)
    src = orc.make_source(kind=1, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5)
    A, B, C = orc.kappa_coeffs(0.3, 0.7, 1, boxes, z, 8, src)
    npix = counts.shape[1]
    k64 = (A[:, None] * counts).sum(0) - C
    ident = (A * counts.sum(1)).sum() / npix - C
    scale = np.abs(A).max() * counts.sum(0).max() + abs(C)
    assert abs(k64.mean() - ident) < 1e-12 * scale
    A0, B0, C0 = orc.kappa_coeffs(0.0, 0.7, 1, boxes, z, 8, src)
    assert np.all(orc.kappa_map(counts, A0, C0) == 0.0)     # no matter, no lensing


@pytest.mark.parametrize("kind,units", [(0, 1), (1, 1), (1, 0)])
def test_complex_step_matches_central_difference(orc, kind, units):
    counts, z, boxes = _small_map(orc, nside=4, nshell=3)
    src = orc.make_source(kind=kind, z_s=1.1, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5)
    rng = np.random.default_rng(4)
    g = rng.normal(size=counts.shape[1]).astype(np.float32)
    th = [0.3, 0.7, 2.0, 1.5, 0.5]
    G = orc.kappa_stat_grads(counts, 4, th[0], th[1], units, boxes, z, src, g)

    def stats(t):
        s = orc.make_source(kind=kind, z_s=1.1, alpha=t[2], beta=t[3], z0=t[4], z_max=1.5)
        return orc.kappa_stats_f64(counts, 4, t[0], t[1], units, boxes, z, s, g)

    # fourth-order central difference (truncation ~ (1e-3)^4, round-off ~ 1e-12)
    for j in range(5):
        h = 1e-3 * th[j]

        def at(k):
            t = list(th)
            t[j] += k * h
            return stats(t)
        fd = (8 * (at(1) - at(-1)) - (at(2) - at(-2))) / (12 * h)
        for s in range(3):
            scale = np.abs(G[s]).max()
            assert G[s, j] == pytest.approx(fd[s], rel=1e-7, abs=1e-8 * scale)
    if units == 1:
        assert np.all(G[:, 1] == 0.0)      # h cancels for lengths in Mpc/h
    else:
        assert np.any(G[:, 1] != 0.0)
    if kind == 0:
        assert np.all(G[:, 2:] == 0.0)     # a source plane has no n(z) parameters


# ---- pins of the unrounded FP64 statistics behind the gradient parity ----
# (var = mu2 as the reading of Eq. 12, skew = mu3 / mu2^(3/2), and
# <g, kappa> with kappa_p = sum_b A_b n_bp - C of Eq. 6)

@pytest.mark.parametrize("kind,units", [(0, 1), (1, 1), (1, 0)])
def test_f64_stats_against_numpy_and_scipy(orc, kind, units):
    """var and skew against numpy / scipy.stats (population definitions,
    an independent library), <g, kappa> against a numpy dot product of the
    map built from the oracle's coefficients (which carry their own pins)."""
    stats = pytest.importorskip("scipy.stats")
    counts, z, boxes = _small_map(orc, nside=4, nshell=3, seed=11)
    src = orc.make_source(kind=kind, z_s=1.1, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5)
    rng = np.random.default_rng(12)
    g = rng.normal(size=counts.shape[1]).astype(np.float32)
    A, B, C = orc.kappa_coeffs(0.3, 0.7, units, boxes, z, 4, src)
    k = counts.astype(np.float64).T @ A - C
    var, skew, gk = orc.kappa_stats_f64(counts, 4, 0.3, 0.7, units, boxes, z, src, g)
    assert var == pytest.approx(np.var(k), rel=1e-12)
    assert skew == pytest.approx(stats.skew(k, bias=True), rel=1e-11)
    assert gk == pytest.approx(float(np.dot(g.astype(np.float64), k)),
                               rel=1e-12, abs=1e-12 * float(np.abs(g).sum() * np.abs(k).max()))
    # the map's -C shifts <g, kappa> by -C sum g, but neither var nor skew
    ones = np.ones_like(g)
    _, _, s1 = orc.kappa_stats_f64(counts, 4, 0.3, 0.7, units, boxes, z, src, ones)
    ident = float((A * counts.sum(1)).sum()) - counts.shape[1] * C
    assert s1 == pytest.approx(ident, rel=1e-12, abs=1e-12 * abs(C) * counts.shape[1])


def test_f64_stats_one_nonzero_pixel_closed_form(orc):
    """Hand-computed case: at Nside 1 (12 pixels) only pixel 0 holds
    particles (20000 in shell 0, 10000 in shell 1, so that a is of the order
    of C and the deviations lose no digits), so kappa takes a - C there and
    -C elsewhere, a = 20000 A_0 + 10000 A_1.  Then mu2 = 11 a^2 / 144 and
    skew = (N - 2) / sqrt(N - 1) = 10 / sqrt(11), whatever C is;
    <1, kappa> = a - 12 C.  A divisor N - 1, a skew without the 3/2 power or
    a dropped -C fails one of these."""
    counts = np.zeros((2, 12), np.int32)
    counts[0, 0], counts[1, 0] = 20000, 10000
    z = np.array([0.3, 0.5, 0.7])
    boxes = [orc.make_box(2000.0, [1000.0] * 3, 64 ** 3, 0, 2)]
    src = orc.make_source(kind=0, z_s=1.2)
    A, B, C = orc.kappa_coeffs(0.3, 0.7, 1, boxes, z, 1, src)
    a = 20000 * A[0] + 10000 * A[1]
    assert 0.1 < a / C < 10
    var, skew, s1 = orc.kappa_stats_f64(counts, 1, 0.3, 0.7, 1, boxes, z, src,
                                        np.ones(12, np.float32))
    assert var == pytest.approx(11 * a * a / 144, rel=1e-14)
    assert skew == pytest.approx(10 / np.sqrt(11), rel=1e-13)
    assert s1 == pytest.approx(a - 12 * C, rel=1e-13)


def test_f64_stats_h_independent_in_mpc_over_h(orc):
    """Lengths in Mpc/h: c/H0 = 2997.92458 Mpc/h carries no h, so every
    coefficient and hence every statistic is the same at any h; in Mpc they
    change with h (the map is then evaluated directly from the coefficients)."""
    counts, z, boxes = _small_map(orc, nside=4, nshell=3, seed=5)
    src = orc.make_source(kind=1, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5)
    g = np.linspace(-1, 1, counts.shape[1]).astype(np.float32)
    a = orc.kappa_stats_f64(counts, 4, 0.3, 0.7, 1, boxes, z, src, g)
    b = orc.kappa_stats_f64(counts, 4, 0.3, 0.55, 1, boxes, z, src, g)
    assert np.array_equal(a, b)
    c = orc.kappa_stats_f64(counts, 4, 0.3, 0.55, 0, boxes, z, src, g)
    A, B, C = orc.kappa_coeffs(0.3, 0.55, 0, boxes, z, 4, src)
    k = counts.astype(np.float64).T @ A - C
    assert c[0] == pytest.approx(np.var(k), rel=1e-12)
    assert abs(c[0] - a[0]) > 1e-3 * a[0]
