"""Pins of the oracle's shell assignment and binning (Eq. 5, Eq. 8, nesting
of Sec. 2.4): count conservation against an independent numpy radius count,
nesting, replication, invalid inputs and the half-open edge rule."""
import numpy as np
import pytest

from paper_1801_05745_gb300 import synth


def _radius_counts(xyz, obs, chi):
    d = xyz.astype(np.float64) - np.asarray(obs)[None, :]
    r = np.sqrt((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2])
    b = np.searchsorted(chi, r, side="right") - 1
    ok = (b >= 0) & (b < len(chi) - 1)
    return np.bincount(b[ok], minlength=len(chi) - 1)


def test_count_conservation_per_shell(orc):
    xyz = synth.particles_numpy(200_000, 2000.0, 5.0, synth.seed_for(9, 0, 0))
    chi = np.linspace(300.0, 990.0, 13)
    box = orc.make_box(2000.0, [1000.0] * 3, 200_000, 0, 12)
    counts, inv = orc.bin_counts(xyz, box, chi, 16)
    assert inv == 0
    assert np.array_equal(counts.sum(1), _radius_counts(xyz, [1000.0] * 3, chi))


def test_keys_match_bin(orc):
    xyz = synth.particles_numpy(50_000, 2000.0, 5.0, synth.seed_for(9, 1, 0))
    chi = np.linspace(100.0, 1000.0, 7)
    box = orc.make_box(2000.0, [1000.0] * 3, 50_000, 0, 6)
    counts, _ = orc.bin_counts(xyz, box, chi, 32)
    k = orc.keys(xyz, box, chi, 32)
    ref = np.bincount(k[k >= 0], minlength=counts.size).reshape(counts.shape)
    assert np.array_equal(counts, ref)
    # pixel part of the key equals the HEALPix pixel of the FP64 vector
    sel = np.nonzero(k >= 0)[0][:2000]
    d = xyz[sel].astype(np.float64) - 1000.0
    assert np.array_equal(k[sel] % (12 * 32 * 32), orc.vec2pix_many(32, d))


def test_nesting_boxes_own_their_shells(orc):
    x1 = synth.particles_numpy(60_000, 2000.0, 5.0, 11)
    x2 = synth.particles_numpy(60_000, 6400.0, 20.0, 12)
    chi = np.array([200.0, 600.0, 1000.0, 2000.0, 3000.0])
    b1 = orc.make_box(2000.0, [1000.0] * 3, 60_000, 0, 2)
    b2 = orc.make_box(6400.0, [3200.0] * 3, 60_000, 2, 4)
    c = np.zeros((4, 12 * 8 * 8), np.int32)
    orc.bin_counts(x1, b1, chi, 8, c)
    orc.bin_counts(x2, b2, chi, 8, c)
    r1 = _radius_counts(x1, [1000.0] * 3, chi)
    r2 = _radius_counts(x2, [3200.0] * 3, chi)
    assert np.array_equal(c.sum(1), np.concatenate([r1[:2], r2[2:]]))


def test_replication_equals_sum_of_shifted_observers(orc):
    """With L and the observer exactly representable, the image (i,j,k) of a
    periodic box is the un-replicated box seen from obs - (i,j,k) L."""
    L = 500.0
    xyz = synth.particles_numpy(3000, L, 5.0, 13)
    chi = np.linspace(200.0, 700.0, 6)
    box = orc.make_box(L, [250.0] * 3, 3000, 0, 5, replicate=1)
    c1, inv = orc.bin_counts(xyz, box, chi, 4)
    c2 = np.zeros_like(c1)
    for i in (-1, 0, 1):
        for j in (-1, 0, 1):
            for k in (-1, 0, 1):
                b = orc.make_box(L, [250.0 - i * L, 250.0 - j * L, 250.0 - k * L], 3000, 0, 5)
                orc.bin_counts(xyz, b, chi, 4, c2)
    assert inv == 0 and np.array_equal(c1, c2) and c1.sum() > 0


def test_half_open_edges_and_invalid(orc):
    chi = np.array([1.0, 2.0, 3.0])
    box = orc.make_box(10.0, [0.0, 0.0, 0.0], 10, 0, 2)
    xyz = np.array([[1.0, 0, 0], [2.0, 0, 0], [3.0, 0, 0], [0.5, 0, 0],
                    [0, 0, 0], [np.nan, 1, 1], [np.inf, 0, 0], [0, 2.5, 0]], np.float32)
    k = orc.keys(xyz, box, chi, 1)
    npix = 12
    assert k[0] // npix == 0 and k[1] // npix == 1   # r == chi_b goes to shell b
    assert k[2] == -1 and k[3] == -1                 # r == chi_S and r < chi_0 dropped
    assert k[4] == -2 and k[5] == -2 and k[6] == -2  # r == 0, NaN, inf invalid
    assert k[7] // npix == 1 and k[7] % npix == 5    # (0, 2.5, 0): phi = pi/2 -> pixel 5
    c, inv = orc.bin_counts(xyz, box, chi, 1)
    assert inv == 3 and c.sum() == 3


def test_openmp_binning_equals_serial(orc):
    """The oracle's all-cores binning (OpenMP, atomic increments) gives the
    serial oracle's counts and invalid count, with and without periodic
    images, non-finite particles included."""
    from paper_1801_05745_gb300 import synth
    x = synth.particles_numpy(120_000, 2000.0, 5.0, synth.seed_for(13, 0, 0))
    x[::997] = np.nan
    chi = orc.chi_edges(0.3, 0.7, 1, np.linspace(0.05, 0.35, 13))
    for R, L in ((0, 2000.0), (1, 500.0)):
        xx = (x % L).astype(np.float32) if R else x
        b = orc.make_box(L, [L / 2] * 3, len(xx), 0, 12, R)
        ref, inv = orc.bin_counts(xx, b, chi, 32)
        got, inv2, threads = orc.bin_counts_omp(xx, b, chi, 32)
        assert np.array_equal(got, ref) and inv == inv2 and threads >= 1
