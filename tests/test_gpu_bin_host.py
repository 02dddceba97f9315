"""Binning from host memory (ufc_bin_host): the positions are copied to the
device in chunks on a second stream while the fast stage runs on the chunks
already copied.  The counts must equal the oracle's (small case, pageable
input) and the device-input path's (boxes spanning several chunks with a
ragged last chunk, page-locked input), bit for bit."""
import numpy as np
import pytest

from paper_1801_05745_gb300 import synth
from tests.gpu_common import api_ctx, both_boxes, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HOST_CHUNK = 1 << 25          # particles per staged chunk in the library


def _nested(orc, nshell):
    z = np.linspace(0.1, 1.5, nshell + 1)
    chi = orc.chi_edges(0.3, 0.7, 1, z)
    return chi, int(np.argmin(np.abs(chi - 1000.0)))


def test_host_input_matches_oracle(orc):
    """Nested boxes, Nside 256, 40 shells, pageable numpy input."""
    api, ctx = api_ctx()
    n = 800_000
    x1 = synth.particles_numpy(n, 2000.0, 5.0, synth.seed_for(2, 3, 0))
    x2 = synth.particles_numpy(n, 6400.0, 20.0, synth.seed_for(2, 3, 1))
    chi, split = _nested(orc, 40)
    b1a, b1o = both_boxes(api, orc, 2000.0, [1000.0] * 3, n, 0, split)
    b2a, b2o = both_boxes(api, orc, 6400.0, [3200.0] * 3, n, split, 40)
    got = ctx.bin_host([x1, x2], [b1a, b2a], chi, 256)
    ctx.synchronize()
    got = got.cpu().numpy()
    ref = np.zeros_like(got)
    orc.bin_counts(x1, b1o, chi, 256, ref)
    orc.bin_counts(x2, b2o, chi, 256, ref)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("nside", [64, 1024])
def test_host_input_chunks_match_device_input(orc, nside):
    """Inner box of 2 chunks + a ragged tail (not a multiple of 4 particles),
    outer box of one partial chunk; both output paths (Nside 64: L2
    atomics, Nside 1024: dense keys)."""
    api, ctx = api_ctx()
    dev = torch.device("cuda", 0)
    n1, n2 = 2 * HOST_CHUNK + 12_345_677, 3_000_001
    x1 = synth.particles_torch(n1, 2000.0, 5.0, synth.seed_for(3, 7, 0), device=dev)
    x2 = synth.particles_torch(n2, 6400.0, 20.0, synth.seed_for(3, 7, 1), device=dev)
    chi, split = _nested(orc, 60)
    b1 = api.make_box(2000.0, [1000.0] * 3, n1, 0, split)
    b2 = api.make_box(6400.0, [3200.0] * 3, n2, split, 60)
    ref = ctx.bin([x1, x2], [b1, b2], chi, nside).clone()
    info_ref = ctx.bin_info()
    h1 = torch.empty(x1.shape, dtype=torch.float32, pin_memory=True)
    h2 = torch.empty(x2.shape, dtype=torch.float32, pin_memory=True)
    h1.copy_(x1)
    h2.copy_(x2)
    torch.cuda.synchronize()
    for _ in range(2):                       # second call reuses the staging buffer
        got = ctx.bin_host([h1, h2], [b1, b2], chi, nside)
        info = ctx.bin_info()
        assert torch.equal(got, ref)
        assert info == info_ref
    assert info["keyed"] == int(ref.sum())


def test_host_input_rejects_bad_arguments(orc):
    api, ctx = api_ctx()
    chi, split = _nested(orc, 10)
    b = api.make_box(2000.0, [1000.0] * 3, 10, 0, 10)
    with pytest.raises(TypeError):
        ctx.bin_host([to_dev(np.zeros((10, 3), np.float32))], [b], chi, 64)
    with pytest.raises(api.UfcError):
        ctx.bin_host([np.zeros((10, 3), np.float32)], [b], chi, 63)


def test_host_input_periodic_images(orc):
    """64^3 particles of a 500 Mpc/h box with 4 image layers (729 images per
    particle: the pending lists drain after every pass) from host memory."""
    api, ctx = api_ctx()
    from paper_1801_05745_gb300 import synth as sy
    L = 500.0
    xyz = sy.particles_numpy(64 ** 3, L, 5.0, sy.seed_for(1, 1, 0))
    c0, c1 = orc.comoving_distance(0.3, 0.7, 1, 0.1), orc.comoving_distance(0.3, 0.7, 1, 0.5)
    chi = np.linspace(c0, c1, 11)
    ba, bo = both_boxes(api, orc, L, [L / 2] * 3, len(xyz), 0, 10, R=4)
    got = ctx.bin_host([xyz], [ba], chi, 64)
    ctx.synchronize()
    ref, inv = orc.bin_counts(xyz, bo, chi, 64)
    assert np.array_equal(got.cpu().numpy(), ref)


@pytest.mark.parametrize("nside", [64, 1024])
def test_streamed_host_input_matches_device_input(orc, nside):
    """ufc_bin_host_stream with 300k-particle chunks (7 chunks over two boxes,
    ragged ends) equals binning the device copies in one call; a second call
    with accumulation (and another chunk size) doubles the counts exactly.
    Nside 64: L2-atomic path; Nside 1024: dense-key path."""
    api, ctx = api_ctx()
    n1, n2 = 1_100_003, 700_001
    x1 = synth.particles_numpy(n1, 2000.0, 5.0, synth.seed_for(2, 5, 0))
    x2 = synth.particles_numpy(n2, 6400.0, 20.0, synth.seed_for(2, 5, 1))
    chi, split = _nested(orc, 60)
    b1 = api.make_box(2000.0, [1000.0] * 3, n1, 0, split)
    b2 = api.make_box(6400.0, [3200.0] * 3, n2, split, 60)
    ref = ctx.bin([to_dev(x1), to_dev(x2)], [b1, b2], chi, nside).clone()
    h1 = torch.from_numpy(x1).pin_memory()
    h2 = torch.from_numpy(x2).pin_memory()
    got = ctx.bin_host_stream([h1, h2], [b1, b2], chi, nside, chunk=300_000)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    ctx.bin_host_stream([h1, h2], [b1, b2], chi, nside, chunk=450_000, counts=got, accumulate=True)
    torch.cuda.synchronize()
    assert torch.equal(got, 2 * ref)
