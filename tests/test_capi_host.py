"""C-ABI checks that need no GPU: the library loads, exports every symbol
the header declares, and its host cosmology (Eq. 1-3, 6) agrees with the
independent oracle."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ufalcon.h")


@pytest.fixture(scope="module")
def api():
    from paper_1801_05745_gb300 import build
    build.build()
    from paper_1801_05745_gb300 import api as a
    return a


def test_header_symbols_exported(api):
    text = open(HEADER).read()
    names = sorted(set(re.findall(r"\b(ufc_[a-z_0-9]+)\s*\(", text)))
    assert len(names) >= 15
    import ctypes
    lib = ctypes.CDLL(api.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_chi_edges_vs_oracle(api, orc):
    z = np.linspace(0.1, 1.5, 61)
    for om, units in [(0.3, 1), (0.276, 1), (1.0, 1), (0.3, 0)]:
        got = api.chi_edges(api.make_cosmo(om, 0.7, units), z)
        ref = orc.chi_edges(om, 0.7, units, z)
        assert np.allclose(got, ref, rtol=1e-13, atol=0)


def test_z_of_chi_vs_oracle(api, orc):
    cosmo = api.make_cosmo(0.3, 0.7, 1)
    chi = np.linspace(292.0, 1322.0, 11)
    got = api.z_of_chi(cosmo, chi)
    ref = np.array([orc.z_of_chi(0.3, 0.7, 1, c) for c in chi])
    assert np.allclose(got, ref, rtol=1e-12)


@pytest.mark.parametrize("kind", [0, 1])
def test_kappa_coeffs_vs_oracle(api, orc, kind):
    z = np.linspace(0.1, 1.5, 21)
    boxes_a = [api.make_box(2000.0, [1000.0] * 3, 512 ** 3, 0, 8),
               api.make_box(6400.0, [3200.0] * 3, 512 ** 3, 8, 20)]
    boxes_o = [orc.make_box(2000.0, [1000.0] * 3, 512 ** 3, 0, 8),
               orc.make_box(6400.0, [3200.0] * 3, 512 ** 3, 8, 20)]
    kw = dict(kind=kind, z_s=1.5, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5)
    A, B, C = api.kappa_coeffs(api.make_cosmo(0.3, 0.7, 1), boxes_a, z, 512, api.make_source(**kw))
    Ao, Bo, Co = orc.kappa_coeffs(0.3, 0.7, 1, boxes_o, z, 512, orc.make_source(**kw))
    assert np.allclose(A, Ao, rtol=1e-12, atol=0)
    assert np.allclose(B, Bo, rtol=1e-12, atol=0)
    assert C == pytest.approx(Co, rel=1e-12)


@pytest.mark.parametrize("kind,units", [(0, 1), (1, 1), (1, 0)])
def test_coefficient_derivatives_vs_oracle_complex_step(api, orc, kind, units):
    """Dual-number dA/dtheta, dC/dtheta against the oracle's complex-step
    gradient of <g, kappa> with g = e_p picking single shells."""
    z = np.linspace(0.2, 1.0, 4)
    nside = 2
    npix = 48
    kw = dict(kind=kind, z_s=1.1, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5)
    boxes_a = [api.make_box(2000.0, [1000.0] * 3, 64 ** 3, 0, 3)]
    boxes_o = [orc.make_box(2000.0, [1000.0] * 3, 64 ** 3, 0, 3)]
    A, B, C, dA, dC = api.kappa_coeffs(api.make_cosmo(0.3, 0.7, units), boxes_a, z, nside,
                                       api.make_source(**kw), derivs=True)
    # counts: one particle in shell b at pixel b; g = indicator of pixel b
    for b in range(3):
        counts = np.zeros((3, npix), np.int32)
        counts[b, b] = 1
        g = np.zeros(npix, np.float32)
        g[b] = 1.0
        G = orc.kappa_stat_grads(counts, nside, 0.3, 0.7, units, boxes_o, z, orc.make_source(**kw), g)
        # <g, kappa> = A_b - C  ->  d/dtheta = dA_b - dC
        assert np.allclose(G[2], dA[:, b] - dC, rtol=1e-11, atol=1e-14 * np.abs(dA).max())


@pytest.mark.parametrize("units", [1, 0])
def test_delta_coeffs_vs_oracle(api, orc, units):
    """Overdensity coefficients (Eq. 7) of the host library against the
    oracle, and their dual-number derivatives against 4th-order central
    differences of the oracle in (Omega_m, h)."""
    z = np.linspace(0.1, 1.5, 21)
    boxes_a = [api.make_box(2000.0, [1000.0] * 3, 512 ** 3, 0, 8),
               api.make_box(6400.0, [3200.0] * 3, 512 ** 3, 8, 20)]
    boxes_o = [orc.make_box(2000.0, [1000.0] * 3, 512 ** 3, 0, 8),
               orc.make_box(6400.0, [3200.0] * 3, 512 ** 3, 8, 20)]
    A, C, dA, dC = api.delta_coeffs(api.make_cosmo(0.3, 0.7, units), boxes_a, z, 256, derivs=True)
    Ao, Co = orc.delta_coeffs(0.3, 0.7, units, boxes_o, z, 256)
    assert np.allclose(A, Ao, rtol=1e-12, atol=0)
    assert C == Co == 1.0
    assert np.all(dC == 0.0) and np.all(dA[2:] == 0.0)     # n(z) parameters do not enter
    for j, (om, h) in enumerate([(1, 0), (0, 1)]):
        e = 1e-3
        f = lambda t: orc.delta_coeffs(0.3 + om * t, 0.7 + h * t, units, boxes_o, z, 256)[0]
        fd = (-f(2 * e) + 8 * f(e) - 8 * f(-e) + f(-2 * e)) / (12 * e)
        assert np.allclose(dA[j], fd, rtol=2e-8, atol=1e-10 * np.abs(A).max())


def test_volume_reading_coeffs_vs_oracle(api, orc):
    """density_volume = 1: kappa and delta coefficients of the host library
    against the oracle, derivatives against central differences."""
    z = np.linspace(0.1, 1.5, 21)
    boxes_a = [api.make_box(2000.0, [1000.0] * 3, 512 ** 3, 0, 8),
               api.make_box(6400.0, [3200.0] * 3, 512 ** 3, 8, 20)]
    boxes_o = [orc.make_box(2000.0, [1000.0] * 3, 512 ** 3, 0, 8),
               orc.make_box(6400.0, [3200.0] * 3, 512 ** 3, 8, 20)]
    kw = dict(kind=1, z_s=1.5, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5)
    cosmo = api.make_cosmo(0.3, 0.7, 1, density_volume=1)
    A, B, C, dA, dC = api.kappa_coeffs(cosmo, boxes_a, z, 512, api.make_source(**kw), derivs=True)
    Ao, Bo, Co = orc.kappa_coeffs(0.3, 0.7, 1, boxes_o, z, 512, orc.make_source(**kw), dens_volume=1)
    assert np.allclose(A, Ao, rtol=1e-12, atol=0) and np.allclose(B, Bo, rtol=1e-12, atol=0)
    assert C == pytest.approx(Co, rel=1e-12)
    e = 1e-3
    f = lambda t: orc.kappa_coeffs(0.3 + t, 0.7, 1, boxes_o, z, 512, orc.make_source(**kw),
                                   dens_volume=1)[0]
    fd = (-f(2 * e) + 8 * f(e) - 8 * f(-e) + f(-2 * e)) / (12 * e)
    assert np.allclose(dA[0], fd, rtol=2e-7, atol=1e-10 * np.abs(A).max())
    Ad, Cd = api.delta_coeffs(cosmo, boxes_a, z, 512)
    Ado, Cdo = orc.delta_coeffs(0.3, 0.7, 1, boxes_o, z, 512, dens_volume=1)
    assert np.allclose(Ad, Ado, rtol=1e-12, atol=0) and Cd == Cdo == 1.0
    with pytest.raises(api.UfcError):
        api.kappa_coeffs(api.make_cosmo(0.3, 0.7, 1, density_volume=2), boxes_a, z, 512,
                         api.make_source(**kw))


def test_grad_from_sums_rejects_bad_input(api):
    """ufc_kappa_grad_from_sums is host-only: it runs without a GPU and
    rejects non-finite sums and sizes it cannot hold (its values are checked
    against the oracle's complex step in tests/test_parallel_gloo.py)."""
    S, nside = 3, 4
    sums = np.ones(4 * S + 4)
    sums[4 * S:] = [0.5, 2.0, 1.0, 0.0]                  # a map with positive variance
    grad, G, H = api.kappa_grad_from_sums(sums, S, nside, np.ones(5 * S), np.zeros(5))
    assert np.all(np.isfinite(grad)) and H == 0.0
    bad = sums.copy()
    bad[5] = np.inf
    with pytest.raises(api.UfcError):
        api.kappa_grad_from_sums(bad, S, nside, np.ones(5 * S), np.zeros(5))
    with pytest.raises(api.UfcError):
        api.kappa_grad_from_sums(sums, S, 3, np.ones(5 * S), np.zeros(5))   # nside not 2^k
