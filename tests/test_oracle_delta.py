"""Pins of the oracle's overdensity-map coefficients (Eq. 7):
delta_p = sum_b [F_b n_bp - Delta chi_b] / sum_b Delta chi_b = sum_b A_b n_bp - C.
Each pin comes from outside the formula: the Einstein-de Sitter closed form
of chi, the geometry of spherical shells for a uniform field, the relation
to the independently computed kappa coefficients of Eq. 6, and scalings."""
import numpy as np
import pytest

C_OVER_H0 = 2997.92458


def _box(orc, L=2000.0, n=64 ** 3, lo=0, hi=10):
    return orc.make_box(L, [L / 2] * 3, n, lo, hi)


def test_delta_eds_closed_form(orc):
    """Omega_m = 1: chi(z) = 2 c/H0 (1 - 1/sqrt(1+z)); then
    A_b = N_pix L^3 / (4 pi N chi_b^2) / (chi_S - chi_0)."""
    z = np.linspace(0.1, 1.5, 11)
    L, n, nside = 2000.0, 64 ** 3, 64
    A, C = orc.delta_coeffs(1.0, 0.7, 1, [_box(orc, L, n)], z, nside)
    chi = 2.0 * C_OVER_H0 * (1.0 - 1.0 / np.sqrt(1.0 + z))
    ref = 12 * nside ** 2 * L ** 3 / (4 * np.pi * n * chi[:-1] ** 2) / (chi[-1] - chi[0])
    assert np.allclose(A, ref, rtol=1e-12, atol=0)
    assert C == 1.0


@pytest.mark.parametrize("nshell", [20, 80])
def test_delta_uniform_field_expectation(orc, nshell):
    """A uniform field of N particles in volume V puts on average
    (N/V) (4 pi / 3)(chi_{b+1}^3 - chi_b^3) / N_pix particles in a pixel of
    shell b.  With F_b at the lower edge the expected delta is then exactly
    sum_b (dchi_b^2 / chi_b + dchi_b^3 / (3 chi_b^2)) / sum_b dchi_b, which
    vanishes to first order in the shell thickness."""
    om, h, nside, L, n = 0.3, 0.7, 128, 3000.0, 10 ** 8
    z = np.linspace(0.1, 1.5, nshell + 1)
    A, C = orc.delta_coeffs(om, h, 1, [_box(orc, L, n, 0, nshell)], z, nside)
    chi = orc.chi_edges(om, h, 1, z)
    npix = 12 * nside ** 2
    mean_counts = (n / L ** 3) * (4 * np.pi / 3) * (chi[1:] ** 3 - chi[:-1] ** 3) / npix
    got = float(np.dot(A, mean_counts) - C)
    d = np.diff(chi)
    ref = float(np.sum(d ** 2 / chi[:-1] + d ** 3 / (3 * chi[:-1] ** 2)) / np.sum(d))
    assert got == pytest.approx(ref, rel=1e-9, abs=1e-13)
    assert 0.0 < got < 2.0 * np.max(d / chi[:-1])


def test_delta_relation_to_kappa_coefficients(orc):
    """Eq. 6 and 7 share F_b: A^kappa_b = 3/2 Om W_b (H0/c) F_b and
    B_b = 3/2 Om W_b (H0/c) dchi_b, so A^kappa_b / A^delta_b = B_b sum dchi / dchi_b."""
    om, h = 0.3, 0.7
    z = np.linspace(0.1, 1.5, 15)
    chi = orc.chi_edges(om, h, 1, z)
    split = 6
    boxes = [orc.make_box(2000.0, [1000.0] * 3, 512 ** 3, 0, split),
             orc.make_box(6400.0, [3200.0] * 3, 512 ** 3, split, 14)]
    src = orc.make_source(kind=1, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5)
    Ak, Bk, Ck = orc.kappa_coeffs(om, h, 1, boxes, z, 256, src)
    Ad, Cd = orc.delta_coeffs(om, h, 1, boxes, z, 256)
    d = np.diff(chi)
    assert np.allclose(Ak / Ad, Bk * d.sum() / d, rtol=1e-11, atol=0)


def test_delta_scalings(orc):
    """A_b scales with V/N of the owning box only; C = 1; in Mpc units
    (lengths c/H0 = 2997.92458/h) A_b carries 1/h for a box whose side is
    held fixed in Mpc."""
    z = np.linspace(0.2, 1.0, 9)
    base, _ = orc.delta_coeffs(0.3, 0.7, 1, [_box(orc, 2000.0, 10 ** 6, 0, 8)], z, 32)
    twice_n, _ = orc.delta_coeffs(0.3, 0.7, 1, [_box(orc, 2000.0, 2 * 10 ** 6, 0, 8)], z, 32)
    twice_l, _ = orc.delta_coeffs(0.3, 0.7, 1, [_box(orc, 4000.0, 10 ** 6, 0, 8)], z, 32)
    assert np.allclose(twice_n, base / 2, rtol=1e-14)
    assert np.allclose(twice_l, base * 8, rtol=1e-14)
    # Mpc units: chi scales by 1/h, so F_b / sum dchi scales by h^3 at fixed L
    mpc, c = orc.delta_coeffs(0.3, 0.7, 0, [_box(orc, 2000.0, 10 ** 6, 0, 8)], z, 32)
    assert np.allclose(mpc, base * 0.7 ** 3, rtol=1e-12)
    assert c == 1.0


@pytest.mark.parametrize("kind", [0, 1])
def test_volume_reading_uniform_field_is_exactly_zero(orc, kind):
    """With the density factor averaged over the shell volume, F_b times the
    expected count of a uniform field is Delta chi_b, so the expected kappa
    (Eq. 6) and delta (Eq. 7) vanish identically; the lower-edge reading
    leaves a positive first-order bias."""
    om, h, nside, L, n = 0.3, 0.7, 64, 3000.0, 10 ** 8
    z = np.linspace(0.1, 1.5, 13)
    chi = orc.chi_edges(om, h, 1, z)
    boxes = [_box(orc, L, n, 0, 12)]
    mean_counts = (n / L ** 3) * (4 * np.pi / 3) * (chi[1:] ** 3 - chi[:-1] ** 3) / (12 * nside ** 2)
    src = orc.make_source(kind=kind, z_s=1.5, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5)
    for vol in (1, 0):
        Ak, _, Ck = orc.kappa_coeffs(om, h, 1, boxes, z, nside, src, dens_volume=vol)
        Ad, Cd = orc.delta_coeffs(om, h, 1, boxes, z, nside, dens_volume=vol)
        ek, ed = float(Ak @ mean_counts - Ck), float(Ad @ mean_counts - Cd)
        if vol:
            assert abs(ek) <= 1e-13 * Ck and abs(ed) <= 1e-13
        else:
            assert ek > 1e-4 * Ck and ed > 1e-4
