"""GPU parity of the fused shell + RING pixel key (Eq. 8, Sec. 2.4
pixelisation): bit-exact against the oracle's FP64 procedure, on seeded
particles, edge-hugging particles and degenerate inputs."""
import numpy as np
import pytest

from paper_1801_05745_gb300 import synth
from tests.gpu_common import api_ctx, boundary_points, both_boxes, to_dev

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nside", [1, 4, 64, 1024])
def test_keys_random_particles(orc, nside):
    api, ctx = api_ctx()
    L = 2000.0
    xyz = synth.particles_numpy(300_000, L, 5.0, synth.seed_for(1, 7, nside % 97))
    chi = orc.chi_edges(0.3, 0.7, 1, np.linspace(0.05, 0.45, 17))
    ba, bo = both_boxes(api, orc, L, [L / 2] * 3, len(xyz), 0, 16)
    got = ctx.keys(to_dev(xyz), ba, chi, nside).cpu().numpy()
    ref = orc.keys(xyz, bo, chi, nside)
    assert np.array_equal(got, ref.astype(np.int32)), np.nonzero(got != ref)[0][:10]
    assert (ref >= 0).sum() > 10_000


@pytest.mark.parametrize("nside", [2, 16, 256, 2048])
def test_keys_on_pixel_and_shell_edges(orc, nside):
    """Directions on pixel edges and radii on shell edges, rounded to FP32:
    exercises the refine and exact stages."""
    api, ctx = api_ctx()
    L = 6400.0
    obs = np.array([3200.0, 3200.0, 3200.0])
    chi = orc.chi_edges(0.3, 0.7, 1, np.linspace(0.1, 0.9, 9))
    d = boundary_points(orc, nside, 40_000, chi[0], chi[-1], seed=nside)
    # radii on shell edges along random directions
    rng = np.random.default_rng(nside + 1)
    u = rng.normal(size=(4000, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    e = chi[rng.integers(0, len(chi), 4000)]
    d = np.concatenate([d, u * e[:, None]])
    # axes, diagonals, poles
    special = []
    for r in (chi[0] * 1.01, chi[3], chi[-1] * 0.99):
        for v in ([1, 0, 0], [0, 1, 0], [-1, 0, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                  [1, 1, 0], [-1, 1, 0], [1, -1, 0.3], [1, 1, 1], [3, 4, 0], [0, 3, 4]):
            v = np.array(v, float)
            special.append(r * v / np.linalg.norm(v))
    d = np.concatenate([d, np.array(special)])
    xyz = (d + obs).astype(np.float32)
    ba, bo = both_boxes(api, orc, L, obs, len(xyz), 0, 8)
    got = ctx.keys(to_dev(xyz), ba, chi, nside).cpu().numpy()
    info = ctx.bin_info()
    ref = orc.keys(xyz, bo, chi, nside)
    bad = np.nonzero(got != ref)[0]
    assert len(bad) == 0, (len(bad), bad[:5], got[bad[:5]], ref[bad[:5]])
    assert info["refined"] > 1000 and info["exact"] > 0, info


def test_keys_degenerate_inputs(orc):
    api, ctx = api_ctx()
    chi = np.array([0.0, 1.0, 2.0, 3.0])
    xyz = np.array([[0, 0, 0], [np.nan, 0, 0], [0, np.inf, 0], [1, 0, 0], [2, 0, 0],
                    [3, 0, 0], [1e-30, 0, 0], [0, 0, 2.5], [0, 0, -2.5],
                    [-0.0, 0.0, 1.5], [0.7, 0.7, 0.0], [-0.7, -0.7, 0.0]], np.float32)
    ba, bo = both_boxes(api, orc, 10.0, [0.0, 0.0, 0.0], 10, 0, 3)
    for nside in (1, 8, 4096):
        got = ctx.keys(to_dev(xyz), ba, chi, nside).cpu().numpy()
        ref = orc.keys(xyz, bo, chi, nside)
        assert np.array_equal(got, ref.astype(np.int32)), (nside, got, ref)
    # empty input
    out = ctx.keys(to_dev(np.zeros((0, 3), np.float32)), ba, chi, 8)
    assert out.numel() == 0


def test_keys_observer_not_representable_in_fp32(orc):
    """An observer with FP64-only coordinates exercises the split shift."""
    api, ctx = api_ctx()
    L = 1000.0
    obs = [500.1234567890123, 499.98765432101234, 500.000000001]
    xyz = synth.particles_numpy(200_000, L, 5.0, 4242)
    chi = np.linspace(50.0, 480.0, 11)
    ba, bo = both_boxes(api, orc, L, obs, len(xyz), 0, 10)
    got = ctx.keys(to_dev(xyz), ba, chi, 128).cpu().numpy()
    ref = orc.keys(xyz, bo, chi, 128)
    assert np.array_equal(got, ref.astype(np.int32))


@pytest.mark.parametrize("path", ["keys", "dense", "direct"])
def test_refine_queue_overflow(orc, path):
    """More undecided particles than the refine stage's queue holds (about
    1/16 of the particles plus one chunk per warp): the overflow takes the
    FP64 procedure inside the fast stage.  25k particles on pixel and shell
    edges, repeated 1000 times: keys and counts equal the oracle's."""
    api, ctx = api_ctx()
    nside, L = 1024, 6400.0
    obs = np.array([3200.0, 3200.0, 3200.0])
    chi = orc.chi_edges(0.3, 0.7, 1, np.linspace(0.1, 0.9, 9))
    d = boundary_points(orc, nside, 20_000, chi[0], chi[-1], seed=77)
    rng = np.random.default_rng(78)
    u = rng.normal(size=(5000, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    d = np.concatenate([d, u * chi[rng.integers(0, len(chi), 5000)][:, None]])
    uniq = (d + obs).astype(np.float32)
    reps = 1000
    xyz = np.tile(uniq, (reps, 1))
    n = len(xyz)
    ba, bo = both_boxes(api, orc, L, obs, n, 0, 8)
    ref = orc.keys(uniq, bo, chi, nside)
    if path == "keys":
        got = ctx.keys(to_dev(xyz), ba, chi, nside).cpu().numpy()
        bad = np.nonzero(got != np.tile(ref, reps))[0]
        assert len(bad) == 0, (len(bad), bad[:5])
    else:
        counts = ctx.bin([to_dev(xyz)], [ba], chi, nside, path=path).cpu().numpy().ravel()
        exp = np.bincount(ref[ref >= 0], minlength=counts.size).astype(np.int64) * reps
        assert np.array_equal(counts.astype(np.int64), exp)
    info = ctx.bin_info()
    cap1 = max(1 << 20, n // 16)
    assert info["refined"] > cap1 // 2, info          # the queue was (nearly) full


def test_paper_shells_at_nside_1024(orc):
    """The paper's own map geometry: 140 shells of dz = 0.01 from z = 0.1 to
    1.5 at Nside 1024 (keys above 2^30).  Keys equal the oracle's; the
    count maps (dense path, 7 GB) hold exactly the oracle's keys."""
    api, ctx = api_ctx()
    nside, nshell, n, L = 1024, 140, 2_000_000, 6400.0
    z = np.array([(10 + b) / 100 for b in range(nshell + 1)])
    chi = orc.chi_edges(0.3, 0.7, 1, z)
    xyz = synth.particles_numpy(n, L, 20.0, synth.seed_for(31, 0, 0))
    ba, bo = both_boxes(api, orc, L, [L / 2] * 3, n, 0, nshell)
    xd = to_dev(xyz)
    got = ctx.keys(xd, ba, chi, nside).cpu().numpy()
    ref = orc.keys(xyz, bo, chi, nside)
    assert np.array_equal(got, ref.astype(np.int32))
    assert ref.max() >= 1 << 30
    counts = ctx.bin([xd], [ba], chi, nside, path="dense").view(-1)
    keys, cnt = np.unique(ref[ref >= 0], return_counts=True)
    assert int(counts.sum()) == int(cnt.sum())
    kt = torch.from_numpy(keys).cuda()
    assert torch.equal(counts[kt].cpu(), torch.from_numpy(cnt.astype(np.int32)))
