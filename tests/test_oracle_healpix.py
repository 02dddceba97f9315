"""Pins of the oracle's HEALPix RING pixelisation (Sec. 2.4 pixelisation),
checked against the published RING geometry, not against the oracle itself."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "healpix_special_points.txt")


def _unit(rng, n):
    p = rng.normal(size=(n, 3))
    return p / np.linalg.norm(p, axis=1)[:, None]


def _centres(orc, nside):
    return np.array([orc.pix2vec(nside, p) for p in range(12 * nside * nside)])


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 64])
def test_roundtrip_all_pixels(orc, nside):
    C = _centres(orc, nside)
    pix = orc.vec2pix_many(nside, C)
    assert np.array_equal(pix, np.arange(12 * nside * nside))


def test_roundtrip_nside1024_sample(orc):
    rng = np.random.default_rng(5)
    p = rng.integers(0, 12 * 1024 * 1024, size=20000)
    p = np.concatenate([p, np.arange(0, 64), 12 * 1024 * 1024 - 1 - np.arange(64),
                        2 * 1024 * 1023 + np.arange(-40, 40)])
    C = np.array([orc.pix2vec(1024, int(q)) for q in p])
    assert np.array_equal(orc.vec2pix_many(1024, C), p)


def test_pixel_centres_follow_ring_geometry(orc):
    # ring heights and azimuths straight from the published formulas
    N = 4
    for pix in range(12 * N * N):
        z, phi = orc.pix2ang(N, pix)
        assert -1 < z < 1 and 0 <= phi < 2 * np.pi
    # the ring of z = 0 is i = 2N with 4N pixels starting at 2N(N-1) + N*4N
    start = 2 * N * (N - 1) + N * 4 * N
    zs = [orc.pix2ang(N, start + j)[0] for j in range(4 * N)]
    assert np.allclose(zs, 0.0, atol=1e-15)


def test_special_directions_golden(orc):
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) >= 10
    for N, x, y, z, p in rows:
        assert orc.vec2pix(int(N), float(x), float(y), float(z)) == int(p), (N, x, y, z)


@pytest.mark.parametrize("nside", [1, 2, 4])
def test_nearest_centre_brute_force(orc, nside):
    """Points well inside a pixel (closer to its centre than 0.3x the minimum
    centre separation) must land in the pixel of the nearest centre."""
    rng = np.random.default_rng(nside)
    C = _centres(orc, nside)
    pts = _unit(rng, 40000)
    pix = orc.vec2pix_many(nside, pts)
    dots = pts @ C.T
    near = dots.argmax(1)
    cc = C @ C.T
    np.fill_diagonal(cc, -2)
    sep = np.arccos(cc.max(1)).min()
    close = np.arccos(np.clip(dots.max(1), -1, 1)) < 0.3 * sep
    assert close.sum() > 4000
    assert np.array_equal(pix[close], near[close])
    # elsewhere most points still agree (HEALPix edges are not bisectors)
    assert (pix == near).mean() > 0.85


@pytest.mark.parametrize("nside", [4, 64])
def test_equal_area_chi2(orc, nside):
    rng = np.random.default_rng(100 + nside)
    npix = 12 * nside * nside
    n = 2_000_000
    pts = _unit(rng, n)
    counts = np.bincount(orc.vec2pix_many(nside, pts), minlength=npix)
    e = n / npix
    chi2 = ((counts - e) ** 2 / e).sum()
    dof = npix - 1
    # 6 sigma band of a chi^2 with dof degrees of freedom
    assert abs(chi2 - dof) < 6 * np.sqrt(2 * dof), (chi2, dof)


def _ring_and_index(N, pix):
    ncap = 2 * N * (N - 1)
    npix = 12 * N * N
    if pix < ncap:
        i = int((1 + np.sqrt(1 + 2 * pix)) // 2)
        while 2 * i * (i - 1) > pix:
            i -= 1
        while 2 * (i + 1) * i <= pix:
            i += 1
        return i, pix - 2 * i * (i - 1), 4 * i
    if pix < npix - ncap:
        k = pix - ncap
        return N + k // (4 * N), k % (4 * N), 4 * N
    q = npix - pix
    i = 1
    while 2 * i * (i + 1) < q:
        i += 1
    return 4 * N - i, pix - (npix - 2 * i * (i + 1)), 4 * i


def _interior(orc, N, pts, eps=1e-9, trials=6, seed=0):
    """Mask of points whose pixel does not change under random 1e-9 nudges."""
    rng = np.random.default_rng(seed)
    base = orc.vec2pix_many(N, pts)
    ok = np.ones(len(pts), bool)
    for _ in range(trials):
        ok &= orc.vec2pix_many(N, pts + eps * rng.normal(size=pts.shape)) == base
    return base, ok


@pytest.mark.parametrize("nside", [1, 2, 8, 64])
def test_quarter_turn_and_mirror_symmetry(orc, nside):
    rng = np.random.default_rng(7 + nside)
    pts = _unit(rng, 20000)
    base, ok = _interior(orc, nside, pts)
    rot = np.stack([-pts[:, 1], pts[:, 0], pts[:, 2]], 1)   # phi -> phi + pi/2
    mir = np.stack([pts[:, 0], pts[:, 1], -pts[:, 2]], 1)   # z -> -z
    prot = orc.vec2pix_many(nside, rot)
    pmir = orc.vec2pix_many(nside, mir)
    checked = 0
    for k in np.nonzero(ok)[0][:5000]:
        i, j, n = _ring_and_index(nside, int(base[k]))
        i2, j2, n2 = _ring_and_index(nside, int(prot[k]))
        assert (i2, n2) == (i, n) and j2 == (j + n // 4) % n
        i3, j3, n3 = _ring_and_index(nside, int(pmir[k]))
        assert i3 == 4 * nside - i and n3 == n
        # mirror keeps phi: same in-ring index
        assert j3 == j
        checked += 1
    assert checked > 1000


def test_azimuth_quarter_turns(orc):
    # exact quadrant axes and diagonal
    assert orc.azimuth_t(1.0, 0.0) == 0.0
    assert orc.azimuth_t(0.0, 1.0) == 1.0
    assert orc.azimuth_t(-1.0, 0.0) == 2.0
    assert orc.azimuth_t(0.0, -1.0) == 3.0
    assert orc.azimuth_t(1.0, 1.0) == 0.5
    assert orc.azimuth_t(-1.0, -1.0) == 2.5
    # against libm atan2 (called, not re-implemented): a few ulp
    rng = np.random.default_rng(3)
    xy = rng.normal(size=(20000, 2))
    ref = np.mod(np.arctan2(xy[:, 1], xy[:, 0]) * (2 / np.pi), 4.0)
    got = np.array([orc.azimuth_t(float(x), float(y)) for x, y in xy])
    assert np.max(np.abs(got - ref)) < 8 * np.finfo(float).eps * 4
