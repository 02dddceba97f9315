"""GPU tests of the batched-realisation call (Sec. 3.2: statistics over many
realisations), the binning-path override used by the autotuner, and the
autograd wrapper of the adjoint."""
import os

import numpy as np
import pytest

from paper_1801_05745_gb300 import synth
from tests.gpu_common import api_ctx, both_boxes, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _realisations(orc, api, nreal, nside, nshell, nbase):
    z = np.linspace(0.1, 1.5, nshell + 1)
    chi = orc.chi_edges(0.3, 0.7, 1, z)
    split = int(np.argmin(np.abs(chi - 1000.0)))
    xs, bxs, As, Cs = [], [], [], []
    src = api.make_source(kind=1, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5)
    for r in range(nreal):
        n1 = synth.poisson_count(nbase, synth.seed_for(4, r, 0))
        n2 = synth.poisson_count(nbase, synth.seed_for(4, r, 1))
        x1 = synth.particles_numpy(n1, 2000.0, 5.0, synth.seed_for(4, r, 0))
        x2 = synth.particles_numpy(n2, 6400.0, 20.0, synth.seed_for(4, r, 1))
        b1 = api.make_box(2000.0, [1000.0] * 3, n1, 0, split)
        b2 = api.make_box(6400.0, [3200.0] * 3, n2, split, nshell)
        A, B, C = api.kappa_coeffs(api.make_cosmo(), [b1, b2], z, nside, src)
        xs.append([to_dev(x1), to_dev(x2)])
        bxs.append([b1, b2])
        As.append(A)
        Cs.append(C)
    return z, chi, xs, bxs, np.array(As), np.array(Cs)


@pytest.mark.parametrize("graph,side_stream,nreal,launches",
                         [(False, True, 5, False), (True, True, 5, False), (True, False, 5, False),
                          (True, True, 19, False), (False, False, 19, False),
                          (False, True, 5, True), (True, True, 19, True), (False, False, 19, True)])
def test_batched_equals_serial(orc, graph, side_stream, nreal, launches):
    """Batched call = the same maps one at a time, bit for bit; with the
    graph on a side stream and on the legacy default stream (captured on
    the context's own stream, joined by events).  Small maps run as one
    persistent kernel, or (launches) on up to 8 concurrent lanes: 19
    realisations use every lane more than once."""
    api, ctx = api_ctx()
    nside, nshell, nb = 64, 12, 100_000
    z, chi, xs, bxs, A, C = _realisations(orc, api, nreal, nside, nshell, nb)
    nbins, lo, hi = 40, -0.05, 0.2
    d = 6 + nbins
    # serial: one call sequence and one synchronisation per realisation
    st_s = api.welford_state(d)
    serial = []
    for r in range(nreal):
        counts = ctx.bin(xs[r], bxs[r], chi, nside)
        _, mom, pdf = ctx.kappa_stats(counts, A[r], C[r], lo, hi, nbins)
        v = ctx.stats_vector(mom, pdf)
        ctx.welford_update(v.view(1, d), st_s)
        torch.cuda.synchronize()
        serial.append((mom.clone(), pdf.clone(), v.clone()))
    st_b = api.welford_state(d)
    torch.cuda.synchronize()
    if side_stream:
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            mom, pdf, stats = ctx.batched_stats(xs, bxs, chi, nside, A, C, lo, hi, nbins, st_b,
                                                graph=graph, launches=launches)
        stream.synchronize()
    else:
        mom, pdf, stats = ctx.batched_stats(xs, bxs, chi, nside, A, C, lo, hi, nbins, st_b,
                                            graph=graph, launches=launches)
        # ordered on the default stream: no explicit synchronisation before use
        mom, pdf, stats = mom.clone(), pdf.clone(), stats.clone()
        torch.cuda.synchronize()
    for r in range(nreal):
        assert torch.equal(mom[r], serial[r][0])
        assert torch.equal(pdf[r], serial[r][1])
        assert torch.equal(stats[r], serial[r][2])
    assert torch.equal(st_b, st_s)             # the same update, in the same order
    mean, cov, corr = ctx.welford_finalize(st_b, d, 1)
    m_o, c_o, r_o = orc.covariance(stats.cpu().numpy(), 1)
    assert np.allclose(cov.cpu().numpy(), c_o, rtol=1e-9, atol=1e-15)


def test_cached_graph_reads_new_data(orc):
    """A repeated graph call with identical arguments relaunches the cached
    graph; refilled particle buffers must give the new realisations'
    statistics (checked against one-at-a-time calls on the new data)."""
    api, ctx = api_ctx()
    nreal, nside, nshell, nb = 4, 64, 10, 80_000
    z, chi, xs, bxs, A, C = _realisations(orc, api, nreal, nside, nshell, nb)
    nbins, lo, hi = 30, -0.05, 0.2
    d = 6 + nbins
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx.batched_stats(xs, bxs, chi, nside, A, C, lo, hi, nbins, api.welford_state(d), graph=True)
    stream.synchronize()
    rng = np.random.default_rng(8)
    for row in xs:                       # new positions in the same buffers
        for x in row:
            perm = torch.from_numpy(rng.permutation(x.shape[0])).cuda()
            x.copy_(torch.roll(x[perm], 1, dims=1))
    torch.cuda.synchronize()
    st_b = api.welford_state(d)
    with torch.cuda.stream(stream):
        mom, pdf, stats = ctx.batched_stats(xs, bxs, chi, nside, A, C, lo, hi, nbins, st_b,
                                            graph=True)
    stream.synchronize()
    for r in range(nreal):
        counts = ctx.bin(xs[r], bxs[r], chi, nside)
        _, m_s, p_s = ctx.kappa_stats(counts, A[r], C[r], lo, hi, nbins)
        torch.cuda.synchronize()
        assert torch.equal(mom[r], m_s) and torch.equal(pdf[r], p_s)


def test_forced_paths_agree_and_autotune(orc, tmp_path, monkeypatch):
    api, ctx = api_ctx()
    from paper_1801_05745_gb300 import autotune
    n = 400_000
    x = synth.particles_numpy(n, 2000.0, 5.0, 31)
    chi = orc.chi_edges(0.3, 0.7, 1, np.linspace(0.1, 0.33, 21))
    b, _ = both_boxes(api, orc, 2000.0, [1000.0] * 3, n, 0, 20)
    xd = to_dev(x)
    c_direct = ctx.bin([xd], [b], chi, 128, path="direct").clone()
    c_dense = ctx.bin([xd], [b], chi, 128, path="dense").clone()
    assert torch.equal(c_direct, c_dense)
    monkeypatch.setenv("UFC_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    p1 = autotune.choose_bin_path(ctx, [xd], [b], chi, 128)
    assert p1 in ("direct", "dense")
    assert os.path.exists(tmp_path / "tune.json")
    assert autotune.choose_bin_path(ctx, [xd], [b], chi, 128) == p1   # cached


@pytest.mark.parametrize("nshell", [10, 140])
def test_autograd_matches_oracle(orc, nshell):
    """Gradients through torch.autograd against the oracle's complex step;
    140 shells (the paper's Delta z = 0.01 from 0.1 to 1.5) take the
    adjoint's launches over two windows of shells."""
    api, ctx = api_ctx()
    from paper_1801_05745_gb300 import autodiff
    nside, n = 32, 300_000
    x1 = synth.particles_numpy(n, 2000.0, 5.0, 61)
    x2 = synth.particles_numpy(n, 6400.0, 20.0, 62)
    z = np.linspace(0.1, 1.5, nshell + 1)
    chi = orc.chi_edges(0.3, 0.7, 1, z)
    split = int(np.argmin(np.abs(chi - 1000.0)))
    b1a, b1o = both_boxes(api, orc, 2000.0, [1000.0] * 3, n, 0, split)
    b2a, b2o = both_boxes(api, orc, 6400.0, [3200.0] * 3, n, split, nshell)
    counts = ctx.bin([to_dev(x1), to_dev(x2)], [b1a, b2a], chi, nside)
    g = torch.from_numpy(np.random.default_rng(2).normal(size=counts.shape[1]).astype(np.float32))
    theta = torch.tensor([0.3, 0.7, 2.0, 1.5, 0.5], dtype=torch.float64, requires_grad=True)
    kap, var, skew = autodiff.kappa_stats(theta, counts, ctx, [b1a, b2a], z, nside)
    loss = 2.0 * var - 0.5 * skew + (kap.double() * g.cuda().double()).sum()
    loss.backward()
    G = orc.kappa_stat_grads(counts.cpu().numpy(), nside, 0.3, 0.7, 1, [b1o, b2o], z,
                             orc.make_source(kind=1, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5),
                             g.numpy())
    ref = 2.0 * G[0] - 0.5 * G[1] + G[2]
    scale = np.abs(2.0 * G[0]).max() + np.abs(0.5 * G[1]).max() + np.abs(G[2]).max()
    assert np.allclose(theta.grad.numpy(), ref, rtol=1e-8, atol=1e-9 * scale)


def test_adjoint_vs_central_difference_step_1e4(orc):
    """Central differences of the oracle's FP64 statistics with step 1e-4
    (counts frozen) agree with the GPU adjoint to the O(h^2) truncation."""
    api, ctx = api_ctx()
    nside, nshell, n = 16, 8, 200_000
    x1 = synth.particles_numpy(n, 2000.0, 5.0, 71)
    x2 = synth.particles_numpy(n, 6400.0, 20.0, 72)
    z = np.linspace(0.1, 1.5, nshell + 1)
    chi = orc.chi_edges(0.3, 0.7, 1, z)
    split = int(np.argmin(np.abs(chi - 1000.0)))
    b1a, b1o = both_boxes(api, orc, 2000.0, [1000.0] * 3, n, 0, split)
    b2a, b2o = both_boxes(api, orc, 6400.0, [3200.0] * 3, n, split, nshell)
    counts = ctx.bin([to_dev(x1), to_dev(x2)], [b1a, b2a], chi, nside)
    cn = counts.cpu().numpy()
    th = np.array([0.3, 0.7, 2.0, 1.5, 0.5])
    A, B, C, dA, dC = api.kappa_coeffs(api.make_cosmo(), [b1a, b2a], z, nside,
                                       api.make_source(kind=1, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5),
                                       derivs=True)
    grad, _, _ = ctx.kappa_backward(counts, A, C, dA, dC, 1.0, 0.0)

    def var_at(t):
        s = orc.make_source(kind=1, alpha=t[2], beta=t[3], z0=t[4], z_max=1.5)
        return orc.kappa_stats_f64(cn, nside, t[0], t[1], 1, [b1o, b2o], z, s)[0]

    for j in (0, 2, 3, 4):
        h = 1e-4 * th[j]
        tp, tm = th.copy(), th.copy()
        tp[j] += h
        tm[j] -= h
        fd = (var_at(tp) - var_at(tm)) / (2 * h)
        assert grad[j] == pytest.approx(fd, rel=1e-6, abs=1e-12)
    assert grad[1] == 0.0


def test_batched_lanes_grow_between_graph_calls(orc):
    """Graph calls on small maps (concurrent lanes): a first call with small
    realisations, then one with ten times the particles, which grows every
    lane's workspace and so drops the cached graph that referred to it; the
    second call rebuilds it and equals the maps computed one at a time."""
    api, ctx = api_ctx()
    nside, nshell, nreal = 64, 12, 11
    nbins, lo, hi = 30, -0.05, 0.2
    d = 6 + nbins
    for nb in (20_000, 200_000):
        z, chi, xs, bxs, A, C = _realisations(orc, api, nreal, nside, nshell, nb)
        st = api.welford_state(d)
        mom, pdf, stats = ctx.batched_stats(xs, bxs, chi, nside, A, C, lo, hi, nbins, st,
                                            graph=True)
        torch.cuda.synchronize()
        for r in range(nreal):
            counts = ctx.bin(xs[r], bxs[r], chi, nside)
            _, m1, p1 = ctx.kappa_stats(counts, A[r], C[r], lo, hi, nbins)
            assert torch.equal(mom[r], m1) and torch.equal(pdf[r], p1)


@pytest.mark.parametrize("chunk,bps", [(1000, 1), (8192, 2), (100_000, 2)])
def test_persistent_batch_tuning_keeps_results(orc, chunk, bps):
    """The persistent kernel's chunk size and blocks per SM (the autotuner's
    choices) change only the speed: every setting gives the serial results
    bit for bit, including realisations whose boxes hold no particle."""
    api, ctx = api_ctx()
    nreal, nside, nshell = 7, 32, 9
    z, chi, xs, bxs, A, C = _realisations(orc, api, nreal, nside, nshell, 30_000)
    xs[3] = [x[:0] for x in xs[3]]             # an empty realisation (its moments are NaN)
    nbins, lo, hi, d = 17, -0.05, 0.2, 6 + 17
    ref = []
    for r in range(nreal):
        counts = ctx.bin(xs[r], bxs[r], chi, nside)
        _, m, p = ctx.kappa_stats(counts, A[r], C[r], lo, hi, nbins)
        ref.append((m.clone(), p.clone()))
    old = ctx.get_tuning()
    try:
        ctx.set_tuning(chunk, bps)
        st = api.welford_state(d)
        mom, pdf, stats = ctx.batched_stats(xs, bxs, chi, nside, A, C, lo, hi, nbins, st, graph=False)
        torch.cuda.synchronize()
    finally:
        ctx.set_tuning(**old)
    for r in range(nreal):       # bit patterns (NaN included)
        assert torch.equal(mom[r].view(torch.int64), ref[r][0].view(torch.int64)), r
        assert torch.equal(pdf[r], ref[r][1]), r
    assert st[0].item() == nreal


def test_batched_run_resumed_from_checkpoint(orc, tmp_path):
    """A batched covariance run stopped after 5 of 12 realisations, saved,
    and resumed in a new context from the checkpoint reaches the state of
    one uninterrupted batched call bit for bit (the updates run in the same
    order)."""
    from paper_1801_05745_gb300 import checkpoint
    api, ctx = api_ctx()
    nside, nshell, nb = 64, 12, 80_000
    z, chi, xs, bxs, A, C = _realisations(orc, api, 12, nside, nshell, nb)
    nbins, lo, hi = 40, -0.05, 0.2
    d = 6 + nbins
    full = api.welford_state(d)
    ctx.batched_stats(xs, bxs, chi, nside, A, C, lo, hi, nbins, full)
    st = api.welford_state(d)
    ctx.batched_stats(xs[:5], bxs[:5], chi, nside, A[:5], C[:5], lo, hi, nbins, st)
    cfg = {"nside": nside, "nshell": nshell, "nbins": nbins, "lo": lo, "hi": hi}
    path = str(tmp_path / "run.npz")
    checkpoint.save(path, st, d, 5, cfg)
    ctx2 = api.Context(0)                        # a context of its own (not the shared one)
    host, k = checkpoint.load(path, d, cfg)
    st2 = torch.from_numpy(host).cuda()
    ctx2.batched_stats(xs[k:], bxs[k:], chi, nside, A[k:], C[k:], lo, hi, nbins, st2)
    torch.cuda.synchronize()
    assert torch.equal(st2, full)
    ctx2.close()
