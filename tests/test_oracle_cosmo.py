"""Pins of the oracle's distances and shell weights (Eq. 1-3, Eq. 6):
closed forms, an independent quadrature library, and limits."""
import numpy as np
import pytest

CH = 2997.92458


@pytest.mark.parametrize("z", [0.05, 0.1, 0.5, 0.8, 1.5, 3.0])
def test_eds_closed_form(orc, z):
    # Omega_m = 1: chi = 2 (c/H0) (1 - 1/sqrt(1+z))
    exact = 2 * CH * (1 - 1 / np.sqrt(1 + z))
    assert orc.comoving_distance(1.0, 0.7, 1, z) == pytest.approx(exact, rel=1e-14)


@pytest.mark.parametrize("z", [0.1, 0.7, 1.5])
def test_de_sitter_limit(orc, z):
    # Omega_m = 0: E = 1, D = z
    assert orc.comoving_distance(0.0, 0.7, 1, z) == pytest.approx(CH * z, rel=1e-14)


def test_lcdm_against_scipy_quad(orc):
    from scipy.integrate import quad
    for om in (0.276, 0.3):
        for z in (0.1, 0.5, 0.8, 1.5):
            ref = quad(lambda x: 1 / np.sqrt(om * (1 + x) ** 3 + 1 - om), 0, z,
                       epsabs=0, epsrel=2e-14, limit=200)[0] * CH
            assert orc.comoving_distance(om, 0.7, 1, z) == pytest.approx(ref, rel=1e-13)


def test_units_mpc_scale_with_h(orc):
    a = orc.comoving_distance(0.3, 0.7, 1, 1.0)
    b = orc.comoving_distance(0.3, 0.7, 0, 1.0)
    assert b == pytest.approx(a / 0.7, rel=1e-15)


def test_z_of_chi_inverts(orc):
    for z in (0.1, 0.37, 1.5):
        chi = orc.comoving_distance(0.3, 0.7, 1, z)
        assert orc.z_of_chi(0.3, 0.7, 1, chi) == pytest.approx(z, rel=1e-13)


def _eds_wb_exact(za, zb, zs):
    """Closed form of Eq. 3 for Omega_m = 1 via the substitution dz/E = dD,
    1 + z = 4/(2 - D)^2: numerator int 4 D (Ds - D)/(Ds (2-D)^2) dD."""
    import sympy as sp
    D, Ds = sp.symbols("D Ds", positive=True)
    f = 4 * D * (Ds - D) / (Ds * (2 - D) ** 2)
    F = sp.integrate(sp.apart(f, D), D)
    d = lambda z: 2 * (1 - 1 / sp.sqrt(sp.Rational(1) + sp.nsimplify(z)))
    Da, Db, Dsv = d(za), d(min(zb, zs)), d(zs)
    num = (F.subs({D: Db, Ds: Dsv}) - F.subs({D: Da, Ds: Dsv}))
    den = d(zb) - Da
    val = complex(sp.N(num / den, 30))
    assert abs(val.imag) < 1e-25   # the log branch terms cancel
    return val.real


@pytest.mark.parametrize("za,zb", [(0.1, 0.11), (0.5, 0.55), (1.2, 1.5), (0.3, 0.9)])
def test_eds_delta_weight_closed_form(orc, za, zb):
    src = orc.make_source(kind=0, z_s=1.5)
    w = orc.shell_weights(1.0, np.array([za, zb]), src)[0]
    assert w == pytest.approx(_eds_wb_exact(za, zb, 1.5), rel=1e-13)


def test_delta_weight_beyond_source_is_zero(orc):
    src = orc.make_source(kind=0, z_s=0.5)
    w = orc.shell_weights(0.3, np.array([0.4, 0.45, 0.5, 0.6]), src)
    assert w[0] > 0 and w[1] > 0 and w[2] == 0.0


def test_thin_shell_limit(orc):
    # Delta z -> 0: W_b -> D (Ds - D)(1+z)/Ds at the shell
    z, dz, zs = 0.7, 1e-4, 1.5
    src = orc.make_source(kind=0, z_s=zs)
    w = orc.shell_weights(0.3, np.array([z - dz / 2, z + dz / 2]), src)[0]
    D = orc.comoving_distance(0.3, 0.7, 1, z) / CH
    Ds = orc.comoving_distance(0.3, 0.7, 1, zs) / CH
    assert w == pytest.approx(D * (Ds - D) * (1 + z) / Ds, rel=1e-7)


def test_nz_weight_against_scipy_nested_quad(orc):
    """n(z) weight against an independent nested quadrature (scipy QUADPACK)."""
    from scipy.integrate import quad
    om, a, b, z0, zmax = 0.3, 2.0, 1.5, 0.5, 1.5
    E = lambda z: np.sqrt(om * (1 + z) ** 3 + 1 - om)
    Dz = lambda z: quad(lambda x: 1 / E(x), 0, z, epsabs=0, epsrel=1e-13)[0]
    n = lambda z: z ** a * np.exp(-(z / z0) ** b)
    norm = quad(n, 0, zmax, epsabs=0, epsrel=1e-13)[0]

    def q(z):
        d = Dz(z)
        return quad(lambda s: n(s) * (Dz(s) - d) / Dz(s), z, zmax, epsabs=0, epsrel=1e-11)[0] / norm

    za, zb = 0.6, 0.65
    num = quad(lambda z: Dz(z) * q(z) * (1 + z) / E(z), za, zb, epsabs=0, epsrel=1e-10)[0]
    den = quad(lambda z: 1 / E(z), za, zb, epsabs=0, epsrel=1e-13)[0]
    src = orc.make_source(kind=1, alpha=a, beta=b, z0=z0, z_max=zmax)
    w = orc.shell_weights(om, np.array([za, zb]), src)[0]
    assert w == pytest.approx(num / den, rel=1e-9)


def test_nz_weight_is_source_average_of_plane_weights(orc):
    """Exchanging the order of integration (Fubini): the n(z) weight equals
    the n(z_s)-weighted average of the single-plane weights W_b(z_s) of
    Eq. 3.  The plane weights are pinned by the EdS closed form above."""
    om, a, b, z0, zmax = 0.3, 2.0, 1.5, 0.5, 1.5
    za, zb = 0.6, 0.65
    n = lambda z: z ** a * np.exp(-(z / z0) ** b)
    x, w = np.polynomial.legendre.leggauss(40)
    num = 0.0
    norm = 0.0
    # W_b(z_s) has kinks at za and zb; n(z) is smooth: split there
    for lo, hi in [(0.0, za), (za, zb), (zb, 1.0), (1.0, zmax)]:
        zs = 0.5 * (hi + lo) + 0.5 * (hi - lo) * x
        wz = 0.5 * (hi - lo) * w
        for s_, ww in zip(zs, wz):
            norm += ww * n(s_)
            if s_ > za:
                wd = orc.shell_weights(om, np.array([za, zb]), orc.make_source(kind=0, z_s=float(s_)))[0]
                num += ww * n(s_) * wd
    src = orc.make_source(kind=1, alpha=a, beta=b, z0=z0, z_max=zmax)
    got = orc.shell_weights(om, np.array([za, zb]), src)[0]
    assert got == pytest.approx(num / norm, rel=1e-10)


def test_kappa_coefficients_structure(orc):
    """A_b, B_b follow Eq. 6: B_b/A_b = Delta chi_b N chi_b^2 4 pi/(N_pix V)."""
    z = np.linspace(0.1, 1.5, 9)
    boxes = [orc.make_box(2000.0, [1000.0] * 3, 512 ** 3, 0, 4),
             orc.make_box(6400.0, [3200.0] * 3, 512 ** 3, 4, 8)]
    src = orc.make_source(kind=0, z_s=1.5)
    A, B, C = orc.kappa_coeffs(0.3, 0.7, 1, boxes, z, 64, src)
    chi = orc.chi_edges(0.3, 0.7, 1, z)
    npix = 12 * 64 * 64
    for b in range(8):
        L = 2000.0 if b < 4 else 6400.0
        ratio = (chi[b + 1] - chi[b]) * 512 ** 3 * chi[b] ** 2 * 4 * np.pi / (npix * L ** 3)
        assert B[b] / A[b] == pytest.approx(ratio, rel=1e-13)
    assert C == pytest.approx(B.sum(), rel=1e-15)
    # the weights enter linearly: A_b = 1.5 Om W_b F_b/(c/H0)
    W = orc.shell_weights(0.3, z, src)
    assert B[2] == pytest.approx(1.5 * 0.3 * W[2] * (chi[3] - chi[2]) / CH, rel=1e-14)
