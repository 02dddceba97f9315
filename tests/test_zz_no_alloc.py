"""GPU test of ufc_kappa_stats_noalloc, the variant of ufc_kappa_stats for
callers that cannot allocate device memory (their memory belongs to another
allocator, or they must not call cudaMalloc once running).  The variant keeps
its scratch in a fixed device array instead of the context workspace; its
results must match the allocating call, on two calls in a row (the second
call reuses the array the first one left behind).

Collected last on purpose (file name), so a failure here does not hide the
other tests in a run that stops at the first failure."""
import ctypes

import numpy as np
import pytest

from paper_1801_05745_gb300 import synth
from tests.gpu_common import api_ctx, both_boxes, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _alloc_outputs(counts, nbins):
    npix = counts.shape[1]
    kap = torch.full((npix,), float("nan"), dtype=torch.float32, device=counts.device)
    mom = torch.full((10,), float("nan"), dtype=torch.float64, device=counts.device)
    pdf = torch.full((nbins + 3,), -1, dtype=torch.int64, device=counts.device)
    return kap, mom, pdf


def _call_noalloc(api, ctx, counts, A, C, lo, hi, nbins, kap, mom, pdf):
    S, npix = counts.shape
    nside = int(round((npix / 12) ** 0.5))
    A = np.ascontiguousarray(A, dtype=np.float64)
    ctx._stream()
    st = api._lib.ufc_kappa_stats_noalloc(ctx.h, ctypes.c_void_p(counts.data_ptr()), S, nside,
                                          A.ctypes.data_as(ctypes.c_void_p), float(C), float(lo),
                                          float(hi), nbins, ctypes.c_void_p(kap.data_ptr()),
                                          ctypes.c_void_p(mom.data_ptr()),
                                          ctypes.c_void_p(pdf.data_ptr()))
    assert st == 0, api._lib.ufc_last_error(ctx.h)


@pytest.mark.parametrize("nside,nshell", [(64, 20), (16, 120)])
def test_noalloc_matches_allocating_call_twice(orc, nside, nshell):
    """The variant runs first, on a fresh context that has never allocated
    its partial-sum workspace: the context's device bytes and the device's
    free memory stay unchanged across both calls; then the allocating call
    on the same context (which does grow its workspace) gives the same map,
    moments and PDF."""
    api, shared = api_ctx()
    n = 300_000
    x1 = synth.particles_numpy(n, 2000.0, 5.0, 8801)
    x2 = synth.particles_numpy(n, 6400.0, 20.0, 8802)
    z = np.linspace(0.1, 1.5, nshell + 1)
    chi = orc.chi_edges(0.3, 0.7, 1, z)
    split = int(np.argmin(np.abs(chi - 1000.0)))
    b1, _ = both_boxes(api, orc, 2000.0, [1000.0] * 3, n, 0, split)
    b2, _ = both_boxes(api, orc, 6400.0, [3200.0] * 3, n, split, nshell)
    counts = shared.bin([to_dev(x1), to_dev(x2)], [b1, b2], chi, nside)
    A, B, C = api.kappa_coeffs(api.make_cosmo(), [b1, b2], z, nside,
                               api.make_source(kind=1, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5))
    ctx = api.Context(0)
    try:
        held0 = ctx.workspace_bytes()
        outs = []
        for i in range(2):
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
            kap, mom, pdf = _alloc_outputs(counts, 64)
            torch.cuda.synchronize()
            free1 = torch.cuda.mem_get_info()[0]
            _call_noalloc(api, ctx, counts, A, C, -0.05, 0.15, 64, kap, mom, pdf)
            torch.cuda.synchronize()
            assert ctx.workspace_bytes() == held0
            if i == 1:   # the first call may load the library's device code
                assert torch.cuda.mem_get_info()[0] == free1, (free0, free1)
            outs.append((kap, mom, pdf))
        kr, mr, pr = ctx.kappa_stats(counts, A, C, -0.05, 0.15, 64)
        torch.cuda.synchronize()
        assert ctx.workspace_bytes() > held0   # the allocating call did allocate
        for kn, mn, pn in outs:
            assert torch.equal(kn, kr)
            assert np.allclose(mn.cpu().numpy(), mr.cpu().numpy(), rtol=1e-12, atol=0)
            assert torch.equal(pn, pr)
    finally:
        ctx.close()


def test_noalloc_rejects_missing_outputs(orc):
    api, ctx = api_ctx()
    counts = torch.zeros((2, 12 * 4 * 4), dtype=torch.int32, device="cuda")
    A = np.ones(2)
    st = api._lib.ufc_kappa_stats_noalloc(ctx.h, ctypes.c_void_p(counts.data_ptr()), 2, 4,
                                          A.ctypes.data_as(ctypes.c_void_p), 0.0, -1.0, 1.0, 8,
                                          None, None, None)
    assert st == 1   # UFC_ERR_ARG
