"""Pins of the oracle's snapshot-mode lightcone (Sec. 2.1: snapshot outputs
spaced 0.02 in redshift; Sec. 2.4: the particles of shell b are those of the
snapshot at the shell's redshift z_b), and the library's host assignment
against it."""
from fractions import Fraction

import numpy as np
import pytest

from paper_1801_05745_gb300 import synth


def test_paper_grid_two_shells_per_snapshot(orc):
    """Shells 0.01 thick from z = 0.1, snapshots 0.02 apart from z = 0.1:
    shell b (z_b = (10 + b)/100) takes snapshot k (z = (10 + 2k)/100) with
    10 + 2k <= 10 + b, i.e. k = floor(b / 2), exact in integers."""
    nshell, nsnap = 140, 71
    z_edges = np.array([float(Fraction(10 + b, 100)) for b in range(nshell + 1)])
    z_snap = np.array([float(Fraction(10 + 2 * k, 100)) for k in range(nsnap)])
    got = orc.snapshot_assign(z_edges, z_snap)
    assert list(got) == [b // 2 for b in range(nshell)]


def test_equal_spacing_is_shell_b_from_snapshot_b(orc):
    """One snapshot per shell at its lower edge: shell b <- snapshot b."""
    z = np.linspace(0.1, 1.5, 61)
    assert list(orc.snapshot_assign(z, z[:-1])) == list(range(60))


def test_grids_built_differently_agree(orc):
    """np.arange and integer-ratio grids differ in the last bits of some
    redshifts; the assignment must not."""
    ze = np.arange(0.1, 1.5 + 1e-9, 0.01)
    zs = np.arange(0.1, 1.5 + 1e-9, 0.02)
    ref = [b // 2 for b in range(len(ze) - 1)]
    assert list(orc.snapshot_assign(ze, zs)) == ref
    ze2 = np.array([(10 + b) / 100 for b in range(len(ze))])
    zs2 = np.array([(10 + 2 * k) / 100 for k in range(len(zs))])
    assert list(orc.snapshot_assign(ze2, zs2)) == ref


def test_shells_below_first_snapshot_are_empty(orc):
    z = np.linspace(0.0, 1.0, 11)
    got = orc.snapshot_assign(z, np.array([0.35, 0.7]))
    assert list(got) == [-1, -1, -1, -1, 0, 0, 0, 1, 1, 1]


def test_single_snapshot_is_the_lightcone_binning(orc):
    """Every shell from one particle set equals binning that set as one box
    owning all shells."""
    n, nshell, nside = 60_000, 12, 16
    x = synth.particles_numpy(n, 2000.0, 5.0, synth.seed_for(11, 0, 0))
    chi = orc.chi_edges(0.3, 0.7, 1, np.linspace(0.05, 0.35, nshell + 1))
    g = orc.make_box(2000.0, [1000.0] * 3, n, 0, nshell)
    got, inv = orc.bin_snapshots([x], [g], np.zeros(nshell, np.int32), chi, nside)
    ref, inv_ref = orc.bin_counts(x, g, chi, nside)
    assert np.array_equal(got, ref) and inv == inv_ref


def test_snapshot_shell_totals_by_radius(orc):
    """Shell b's total equals the number of snapshot s(b)'s particles whose
    FP64 radius (numpy) lies in [chi_b, chi_{b+1}); empty shells stay 0."""
    n, nshell, nside = 50_000, 10, 8
    xs = [synth.particles_numpy(n, 2000.0, 5.0, synth.seed_for(12, 0, k)) for k in range(3)]
    chi = orc.chi_edges(0.3, 0.7, 1, np.linspace(0.05, 0.3, nshell + 1))
    obs = np.array([1000.0] * 3)
    geoms = [orc.make_box(2000.0, obs, n, 0, 1) for _ in xs]
    sos = np.array([-1, 0, 0, 1, 1, 1, 2, -1, 2, 0], np.int32)
    got, inv = orc.bin_snapshots(xs, geoms, sos, chi, nside)
    assert inv == 0
    for b in range(nshell):
        if sos[b] < 0:
            assert got[b].sum() == 0
            continue
        d = xs[sos[b]].astype(np.float64) - obs
        r = np.sqrt((d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2])
        assert got[b].sum() == np.count_nonzero((r >= chi[b]) & (r < chi[b + 1]))


def test_library_assignment_matches_oracle(orc):
    from paper_1801_05745_gb300 import build
    build.build()
    from paper_1801_05745_gb300 import api
    rng = np.random.default_rng(5)
    for _ in range(20):
        ze = np.sort(rng.uniform(0, 2, rng.integers(2, 80)))
        ze = np.unique(ze)
        zs = np.unique(np.sort(rng.uniform(-0.1, 2.1, rng.integers(1, 40))))
        if len(ze) < 2:
            continue
        assert np.array_equal(api.snapshot_assign(ze, zs), orc.snapshot_assign(ze, zs))
    for ze, zs in [(np.array([0.2, 0.1]), np.array([0.0])),
                   (np.array([0.1, 0.2]), np.array([0.1, 0.1])),
                   (np.array([0.1, np.nan]), np.array([0.0]))]:
        with pytest.raises(api.UfcError):
            api.snapshot_assign(ze, zs)
