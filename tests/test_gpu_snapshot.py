"""Snapshot-mode lightcone on the GPU (ufc_bin_snapshots): shell b binned
from the particles of its snapshot (Sec. 2.1, 2.4), bit-exact against the
oracle's shell-by-shell binning.  Also the dense path's shell window (a call
whose boxes own only some shells): the other shells are zeroed when
overwriting and left alone when accumulating."""
import numpy as np
import pytest

from paper_1801_05745_gb300 import synth
from tests.gpu_common import api_ctx, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _snapshots(n, nsnap, L, seed_cfg):
    return [synth.particles_numpy(n + 17 * k, L, 5.0, synth.seed_for(seed_cfg, 0, k))
            for k in range(nsnap)]


@pytest.mark.parametrize("nside,path", [(64, None), (256, "dense"), (256, "direct")])
def test_snapshots_match_oracle(orc, nside, path):
    """10 snapshots 0.02 apart feeding 20 shells 0.01 thick (two shells per
    snapshot), box of 2000 Mpc/h around the observer."""
    api, ctx = api_ctx()
    n, L = 300_000, 2000.0
    z_edges = np.array([(10 + b) / 100 for b in range(21)])
    z_snap = np.array([(10 + 2 * k) / 100 for k in range(10)])
    sos = api.snapshot_assign(z_edges, z_snap)
    assert np.array_equal(sos, orc.snapshot_assign(z_edges, z_snap))
    chi = orc.chi_edges(0.3, 0.7, 1, z_edges)
    xs = _snapshots(n, 10, L, 21)
    geoms_a = [api.make_box(L, [L / 2] * 3, len(x), 0, 1) for x in xs]
    geoms_o = [orc.make_box(L, [L / 2] * 3, len(x), 0, 1) for x in xs]
    counts = torch.full((20, 12 * nside * nside), 7, dtype=torch.int32, device="cuda")
    ctx.bin_snapshots([to_dev(x) for x in xs], geoms_a, sos, chi, nside, counts=counts, path=path)
    ctx.synchronize()
    ref, _ = orc.bin_snapshots(xs, geoms_o, sos, chi, nside)
    assert np.array_equal(counts.cpu().numpy(), ref)


def test_many_runs_several_passes(orc):
    """40 shells alternating between 3 snapshots (40 runs: three passes of
    up to 16), with unassigned shells; then the same call accumulating."""
    api, ctx = api_ctx()
    n, L, nside, S = 200_000, 2000.0, 128, 40
    chi = orc.chi_edges(0.3, 0.7, 1, np.linspace(0.05, 0.33, S + 1))
    xs = _snapshots(n, 3, L, 22)
    sos = np.array([(b % 3) if b % 7 else -1 for b in range(S)], np.int32)
    geoms_a = [api.make_box(L, [L / 2] * 3, len(x), 0, 1) for x in xs]
    geoms_o = [orc.make_box(L, [L / 2] * 3, len(x), 0, 1) for x in xs]
    xd = [to_dev(x) for x in xs]
    for path in (None, "dense"):
        counts = torch.full((S, 12 * nside * nside), -3, dtype=torch.int32, device="cuda")
        ctx.bin_snapshots(xd, geoms_a, sos, chi, nside, counts=counts, path=path)
        ref, _ = orc.bin_snapshots(xs, geoms_o, sos, chi, nside)
        assert np.array_equal(counts.cpu().numpy(), ref)
        ctx.bin_snapshots(xd, geoms_a, sos, chi, nside, counts=counts, accumulate=True, path=path)
        assert np.array_equal(counts.cpu().numpy(), 2 * ref)


def test_no_shell_assigned_zeroes_or_keeps(orc):
    api, ctx = api_ctx()
    chi = orc.chi_edges(0.3, 0.7, 1, np.linspace(0.1, 0.2, 5))
    x = to_dev(_snapshots(1000, 1, 2000.0, 23)[0])
    g = api.make_box(2000.0, [1000.0] * 3, 1000, 0, 1)
    counts = torch.full((4, 12 * 64 * 64), 5, dtype=torch.int32, device="cuda")
    ctx.bin_snapshots([x], [g], np.full(4, -1, np.int32), chi, 64, counts=counts, accumulate=True)
    assert int(counts.min()) == 5 and int(counts.max()) == 5
    ctx.bin_snapshots([x], [g], np.full(4, -1, np.int32), chi, 64, counts=counts)
    assert int(counts.abs().max()) == 0
    with pytest.raises(api.UfcError):
        ctx.bin_snapshots([x], [g], np.array([0, 1, -1, 0], np.int32), chi, 64, counts=counts)


@pytest.mark.parametrize("accumulate", [False, True])
def test_dense_window_leaves_other_shells(orc, accumulate):
    """One box owning shells [5, 9) of 16 at Nside 512 on the dense path:
    shells outside the window are zeroed (overwrite) or unchanged
    (accumulate); inside, the oracle's counts (plus the old values)."""
    api, ctx = api_ctx()
    n, L, nside, S = 1_000_000, 2000.0, 512, 16
    chi = orc.chi_edges(0.3, 0.7, 1, np.linspace(0.05, 0.35, S + 1))
    x = synth.particles_numpy(n, L, 5.0, synth.seed_for(24, 0, 0))
    ba = api.make_box(L, [L / 2] * 3, n, 5, 9)
    bo = orc.make_box(L, [L / 2] * 3, n, 5, 9)
    npix = 12 * nside * nside
    g = torch.Generator(device="cpu").manual_seed(3)
    old = torch.randint(0, 1000, (S, npix), dtype=torch.int32, generator=g)
    counts = old.cuda()
    ctx.bin([to_dev(x)], [ba], chi, nside, counts=counts, accumulate=accumulate, path="dense")
    ref, _ = orc.bin_counts(x, bo, chi, nside)
    got = counts.cpu().numpy()
    exp = ref + (old.numpy() if accumulate else 0)
    assert np.array_equal(got, exp)
    assert ref[:5].sum() == 0 and ref[9:].sum() == 0 and ref[5:9].sum() > 0


@pytest.mark.parametrize("nside,path", [(128, None), (512, "dense")])
def test_snapshots_from_host_memory(orc, nside, path):
    """ufc_bin_snapshots_host streams each run's particles from host memory
    in chunks smaller than a snapshot (ragged last chunk): counts equal
    the device-input call's, and the oracle's, bit for bit."""
    api, ctx = api_ctx()
    n, L = 250_001, 2000.0
    z_edges = np.array([(10 + b) / 100 for b in range(21)])
    z_snap = np.array([(10 + 2 * k) / 100 for k in range(10)])
    sos = api.snapshot_assign(z_edges, z_snap)
    chi = orc.chi_edges(0.3, 0.7, 1, z_edges)
    xs = _snapshots(n, 10, L, 25)
    geoms_a = [api.make_box(L, [L / 2] * 3, len(x), 0, 1) for x in xs]
    geoms_o = [orc.make_box(L, [L / 2] * 3, len(x), 0, 1) for x in xs]
    dev = ctx.bin_snapshots([to_dev(x) for x in xs], geoms_a, sos, chi, nside, path=path).clone()
    host = ctx.bin_snapshots_host(xs, geoms_a, sos, chi, nside, 60_000, path=path)
    ctx.synchronize()
    assert torch.equal(host, dev)
    ref, _ = orc.bin_snapshots(xs, geoms_o, sos, chi, nside)
    assert np.array_equal(host.cpu().numpy(), ref)
