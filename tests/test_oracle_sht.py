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
