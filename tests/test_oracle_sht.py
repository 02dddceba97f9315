"""Pins of the oracle's spherical-harmonic analysis (the full-sky C_l whose
covariance the paper estimates, Sec. 3.2, Eq. 10-11): library values of
Y_lm, exact cases of the pixel sum, exact symmetries of the HEALPix grid,
and the m >= 0 form of C_l against a brute-force sum over all m."""
import numpy as np
import pytest


def _ring_layout(nside):
    """(first pixel, pixel count) of every RING ring, north to south."""
    out, start = [], 0
    for i in range(1, 4 * nside):
        n = 4 * min(i, nside, 4 * nside - i)
        out.append((start, n))
        start += n
    return out


def test_lambda_against_scipy(orc):
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    lmax = 40
    for th in (0.05, 0.7, 1.2, 2.9):
        lam = orc.lambda_lm(np.cos(th), lmax)
        for l in range(lmax + 1):
            for m in range(l + 1):
                ref = sp.sph_harm_y(l, m, th, 0.0).real
                assert lam[orc.alm_index(lmax, l, m)] == pytest.approx(ref, rel=1e-11, abs=1e-13)


def test_constant_map_monopole(orc):
    nside, lmax = 8, 10
    a = orc.map2alm(np.full(12 * nside ** 2, 2.5, np.float32), nside, lmax)
    assert a[orc.alm_index(lmax, 0, 0)] == pytest.approx(2.5 * np.sqrt(4 * np.pi), rel=1e-14)
    cl = orc.alm2cl(a, lmax)
    assert cl[0] == pytest.approx(4 * np.pi * 2.5 ** 2, rel=1e-13)


def test_dipole_of_z_map_against_ring_sum(orc):
    """map_p = z_p: a_10 = (4 pi / N_pix) sqrt(3 / 4 pi) sum_p z_p^2, with the
    sum over rings from the ring heights: polar ring i has 4i pixels at
    z = 1 - i^2/(3N^2), equatorial ring i has 4N at z = 4/3 - 2i/(3N)."""
    nside, lmax = 16, 4
    npix = 12 * nside ** 2
    zmap = np.empty(npix)
    for p in range(npix):
        zmap[p] = orc.pix2ang(nside, p)[0]
    s = 0.0
    for i in range(1, 4 * nside):
        if i < nside:
            z, n = 1 - i * i / (3 * nside ** 2), 4 * i
        elif i <= 3 * nside:
            z, n = 4 / 3 - 2 * i / (3 * nside), 4 * nside
        else:
            k = 4 * nside - i
            z, n = -(1 - k * k / (3 * nside ** 2)), 4 * k
        s += n * z * z
    a = orc.map2alm(zmap.astype(np.float32), nside, lmax)
    ref = 4 * np.pi / npix * np.sqrt(3 / (4 * np.pi)) * s
    assert a[orc.alm_index(lmax, 1, 0)].real == pytest.approx(ref, rel=2e-7)   # FP32 map values


def test_quarter_turn_and_reflection(orc):
    """Rotating the map by a quarter turn (each ring's pixels shifted by a
    quarter of the ring) multiplies a_lm by exp(-i m pi/2); mirroring z -> -z
    (ring i <-> 4N - i) multiplies it by (-1)^(l+m)."""
    nside, lmax = 8, 23
    rng = np.random.default_rng(4)
    m0 = rng.normal(size=12 * nside ** 2).astype(np.float32)
    rings = _ring_layout(nside)
    rot = np.empty_like(m0)
    mir = np.empty_like(m0)
    for (s, n), (s2, n2) in zip(rings, rings[::-1]):
        rot[s:s + n] = np.roll(m0[s:s + n], n // 4)
        mir[s2:s2 + n2] = m0[s:s + n]
    a = orc.map2alm(m0, nside, lmax)
    ar = orc.map2alm(rot, nside, lmax)
    am = orc.map2alm(mir, nside, lmax)
    scale = np.abs(a).max()
    for l in range(lmax + 1):
        for m in range(l + 1):
            k = orc.alm_index(lmax, l, m)
            assert abs(ar[k] - a[k] * np.exp(-0.5j * np.pi * m)) < 1e-12 * scale
            assert abs(am[k] - a[k] * (-1) ** (l + m)) < 1e-12 * scale
    assert np.allclose(orc.alm2cl(ar, lmax), orc.alm2cl(a, lmax), rtol=1e-11)


def test_cl_against_all_m_bruteforce(orc):
    """C_l from m >= 0 (real map: a_l,-m = (-1)^m conj a_lm) against the
    direct sum of |a_lm|^2 over -l <= m <= l with every a_lm computed from
    scipy's Y_lm at the pixel centres."""
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    nside, lmax = 4, 11
    npix = 12 * nside ** 2
    rng = np.random.default_rng(9)
    mp = rng.normal(size=npix).astype(np.float32)
    th = np.empty(npix)
    ph = np.empty(npix)
    for p in range(npix):
        z, phi = orc.pix2ang(nside, p)
        th[p], ph[p] = np.arccos(z), phi
    cl_ref = np.zeros(lmax + 1)
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            a = 4 * np.pi / npix * np.sum(mp * np.conj(sp.sph_harm_y(l, m, th, ph)))
            cl_ref[l] += abs(a) ** 2
        cl_ref[l] /= 2 * l + 1
    cl = orc.alm2cl(orc.map2alm(mp, nside, lmax), lmax)
    assert np.allclose(cl, cl_ref, rtol=1e-10, atol=1e-14 * cl_ref.max())


def test_synthesis_single_modes(orc):
    """a_l0 = 1 gives lambda_l0 = sqrt((2l+1)/4pi) P_l(z) (numpy Legendre);
    a_lm = c (m > 0) gives 2 Re(c Y_lm) (scipy)."""
    nside, lmax = 8, 12
    npix = 12 * nside ** 2
    z = np.array([orc.pix2ang(nside, p)[0] for p in range(npix)])
    ph = np.array([orc.pix2ang(nside, p)[1] for p in range(npix)])
    for l in (0, 1, 5, 12):
        a = np.zeros(orc.alm_size(lmax), complex)
        a[orc.alm_index(lmax, l, 0)] = 1.0
        ref = np.sqrt((2 * l + 1) / (4 * np.pi)) * np.polynomial.legendre.Legendre.basis(l)(z)
        assert np.allclose(orc.alm2map(a, nside, lmax), ref, rtol=1e-12, atol=1e-13)
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    c = 0.7 - 1.3j
    for l, m in ((3, 2), (12, 7), (9, 9)):
        a = np.zeros(orc.alm_size(lmax), complex)
        a[orc.alm_index(lmax, l, m)] = c
        ref = 2 * np.real(c * sp.sph_harm_y(l, m, np.arccos(z), ph))
        assert np.allclose(orc.alm2map(a, nside, lmax), ref, rtol=1e-11, atol=1e-13)


def test_synthesis_real_field_all_m(orc):
    """Random a_lm (m >= 0): the map equals the sum over -l <= m <= l with
    a_l,-m = (-1)^m conj(a_lm), every Y_lm from scipy."""
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    nside, lmax = 4, 10
    npix = 12 * nside ** 2
    rng = np.random.default_rng(6)
    a = rng.normal(size=orc.alm_size(lmax)) + 1j * rng.normal(size=orc.alm_size(lmax))
    for l in range(lmax + 1):
        a[orc.alm_index(lmax, l, 0)] = a[orc.alm_index(lmax, l, 0)].real   # real field: a_l0 real
    th = np.array([np.arccos(orc.pix2ang(nside, p)[0]) for p in range(npix)])
    ph = np.array([orc.pix2ang(nside, p)[1] for p in range(npix)])
    ref = np.zeros(npix, complex)
    for l in range(lmax + 1):
        for m in range(-l, l + 1):
            alm = a[orc.alm_index(lmax, l, abs(m))]
            if m < 0:
                alm = (-1) ** m * np.conj(alm)
            ref += alm * sp.sph_harm_y(l, m, th, ph)
    assert np.abs(ref.imag).max() < 1e-12 * np.abs(ref).max()
    assert np.allclose(orc.alm2map(a, nside, lmax), ref.real, rtol=1e-11, atol=1e-12)


def test_gaussian_beam_is_the_gaussian_kernel(orc):
    """b_l of r.m.s. radius sigma against the Legendre transform of the
    normalised kernel K(g) = exp(-g^2 / 2 sigma^2) / (2 pi sigma^2):
    2 pi int K(g) P_l(cos g) sin g dg, equal to first order in sigma^2."""
    integrate = pytest.importorskip("scipy.integrate")
    sp = pytest.importorskip("scipy.special")
    sigma = 10.8 / 60 * np.pi / 180
    b = orc.gauss_beam(sigma, 1000)
    for l in (0, 10, 100, 500, 1000):
        f = lambda g: (np.exp(-g * g / (2 * sigma ** 2)) / (2 * np.pi * sigma ** 2)
                       * sp.eval_legendre(l, np.cos(g)) * np.sin(g))
        ref = 2 * np.pi * integrate.quad(f, 0.0, 12 * sigma, limit=400, epsabs=1e-14)[0]
        assert b[l] == pytest.approx(ref, rel=2e-3, abs=1e-6)
