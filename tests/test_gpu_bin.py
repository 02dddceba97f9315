"""GPU parity of the per-shell count maps (Eq. 5, Eq. 8, nesting and
replication of Sec. 2.4): bit-exact against the oracle for every output
path (L2 atomics for small maps, the dense scatter + shared-memory histogram
path for large ones), multi-box calls, accumulation and virtual shards."""
import numpy as np
import pytest

from paper_1801_05745_gb300 import synth
from tests.gpu_common import api_ctx, both_boxes, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_tiny_replicated_box(orc):
    """64^3 particles, 500 Mpc/h periodic box, 10 equal-Delta-chi shells
    z = 0.1 - 0.5, Nside 64, 4 image layers."""
    api, ctx = api_ctx()
    L = 500.0
    xyz = synth.particles_numpy(64 ** 3, L, 5.0, synth.seed_for(1, 0, 0))
    c0, c1 = orc.comoving_distance(0.3, 0.7, 1, 0.1), orc.comoving_distance(0.3, 0.7, 1, 0.5)
    chi = np.linspace(c0, c1, 11)
    ba, bo = both_boxes(api, orc, L, [L / 2] * 3, len(xyz), 0, 10, R=4)
    got = ctx.bin([to_dev(xyz)], [ba], chi, 64).cpu().numpy()
    ref, inv = orc.bin_counts(xyz, bo, chi, 64)
    assert inv == 0
    assert np.array_equal(got, ref)
    assert ref.sum() > 10_000_000


@pytest.mark.parametrize("nside,nshell", [(64, 40), (512, 10), (256, 40)])
def test_nested_two_boxes(orc, nside, nshell):
    """Inner 2000 Mpc/h box owning r < 1000, outer 6400 Mpc/h box beyond."""
    api, ctx = api_ctx()
    n = 1_000_000
    x1 = synth.particles_numpy(n, 2000.0, 5.0, synth.seed_for(2, 0, 0))
    x2 = synth.particles_numpy(n, 6400.0, 20.0, synth.seed_for(2, 0, 1))
    z = np.linspace(0.1, 1.5, nshell + 1)
    chi = orc.chi_edges(0.3, 0.7, 1, z)
    split = int(np.argmin(np.abs(chi - 1000.0)))
    b1a, b1o = both_boxes(api, orc, 2000.0, [1000.0] * 3, n, 0, split)
    b2a, b2o = both_boxes(api, orc, 6400.0, [3200.0] * 3, n, split, nshell)
    got = ctx.bin([to_dev(x1), to_dev(x2)], [b1a, b2a], chi, nside)
    info = ctx.bin_info()
    got = got.cpu().numpy()
    ref = np.zeros_like(got)
    orc.bin_counts(x1, b1o, chi, nside, ref)
    orc.bin_counts(x2, b2o, chi, nside, ref)
    assert np.array_equal(got, ref), np.nonzero((got != ref).ravel())[0][:10]
    assert info["keyed"] == ref.sum()


def test_accumulate_and_virtual_shards(orc):
    """Binning K shards with UFC_BIN_ACCUMULATE equals one pass (the
    subvolume decomposition of Sec. 2.4), on both output paths."""
    api, ctx = api_ctx()
    n = 600_000
    x = synth.particles_numpy(n, 2000.0, 5.0, 77)
    chi = orc.chi_edges(0.3, 0.7, 1, np.linspace(0.1, 0.33, 11))
    ba, _ = both_boxes(api, orc, 2000.0, [1000.0] * 3, n, 0, 10)
    for nside in (32, 512):
        one = ctx.bin([to_dev(x)], [ba], chi, nside).clone()
        acc = torch.zeros_like(one)
        for part in np.array_split(x, 5):
            ctx.bin([to_dev(part)], [ba], chi, nside, counts=acc, accumulate=True)
        assert torch.equal(one, acc)


def test_empty_and_invalid_inputs(orc):
    api, ctx = api_ctx()
    chi = np.array([100.0, 200.0, 300.0])
    ba, bo = both_boxes(api, orc, 1000.0, [500.0] * 3, 10, 0, 2)
    c = ctx.bin([to_dev(np.zeros((0, 3), np.float32))], [ba], chi, 16)
    assert int(c.sum()) == 0
    x = np.array([[500, 500, 500], [np.nan, 1, 1], [650, 500, 500]], np.float32)
    c = ctx.bin([to_dev(x)], [ba], chi, 16)
    info = ctx.bin_info()
    ref, inv = orc.bin_counts(x, bo, chi, 16)
    assert np.array_equal(c.cpu().numpy(), ref) and info["invalid"] == inv == 2
    # invalid arguments are rejected before any launch
    from paper_1801_05745_gb300.api import UfcError
    with pytest.raises(UfcError):
        ctx.bin([to_dev(x)], [ba], np.array([100.0, 90.0, 300.0]), 16)
    with pytest.raises(UfcError):
        ctx.bin([to_dev(x)], [ba], chi, 12)


def test_crowded_buckets_wrap_shared_counters(orc):
    """Every particle in two neighbouring pixel blocks of one shell, about
    2 x 65536 per block and CTA: the dense path's shared-memory bucket
    counters hold 16 bits, two to a 32-bit word, so each CTA's counters of
    both halves wrap and carry into the global histogram; the count map
    stays exact (Eq. 5)."""
    api, ctx = api_ctx()
    nside, L = 512, 2000.0
    chi = orc.chi_edges(0.3, 0.7, 1, np.linspace(0.1, 0.33, 11))
    r = 0.5 * (chi[4] + chi[5])
    blk_pix = 24576                         # pixels of one bucket's block
    b0 = 64                                 # an even block: the low halves of a counter word
    pix = np.array([b0 * blk_pix + 100, b0 * blk_pix + 5000,
                    (b0 + 1) * blk_pix + 300, (b0 + 1) * blk_pix + 7000])
    pts = np.array([1000.0 + r * orc.pix2vec(nside, int(p)) for p in pix], np.float32)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = 4 * 65536 * sms                      # ~2 x 65536 per block and CTA (one CTA per SM)
    xyz = np.tile(pts, (n // len(pts), 1))
    n = len(xyz)
    ba, bo = both_boxes(api, orc, L, [L / 2] * 3, n, 0, 10)
    k = orc.keys(pts, bo, chi, nside)
    npix = 12 * nside * nside
    assert np.array_equal(k, 4 * npix + pix)        # the intended shell and pixels
    ref = np.zeros((10, npix), np.int32)
    np.add.at(ref.reshape(-1), k, n // len(pts))
    got = ctx.bin([to_dev(xyz)], [ba], chi, nside, path="dense")
    info = ctx.bin_info()
    assert np.array_equal(got.cpu().numpy(), ref)
    assert info["keyed"] == n
