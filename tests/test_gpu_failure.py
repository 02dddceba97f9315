"""Failure detection without a GPU fault: every device-side wait of the
library is bounded, and a wait that runs out is counted and reported by
ufc_synchronize as UFC_ERR_TIMEOUT, with the context still usable.  The
self-test makes one such wait run out on a barrier that nothing completes."""
import numpy as np
import pytest

from paper_1801_05745_gb300 import synth
from tests.gpu_common import api_ctx, both_boxes, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _small_bin(api, ctx, orc):
    n = 200_000
    x = synth.particles_numpy(n, 2000.0, 5.0, 4242)
    chi = orc.chi_edges(0.3, 0.7, 1, np.linspace(0.1, 0.4, 9))
    ba, bo = both_boxes(api, orc, 2000.0, [1000.0] * 3, n, 0, 8)
    got = ctx.bin([to_dev(x)], [ba], chi, 64)
    ref, inv = orc.bin_counts(x, bo, chi, 64)
    return got, ref


def test_timeout_reported_once_and_context_usable(orc):
    api, ctx = api_ctx()
    ctx.synchronize()                       # nothing pending
    ctx.wait_selftest(1000)
    with pytest.raises(api.UfcError, match="status 4.*bounded wait"):
        ctx.synchronize()
    ctx.synchronize()                       # reported once, then cleared
    got, ref = _small_bin(api, ctx, orc)
    ctx.synchronize()
    assert np.array_equal(got.cpu().numpy(), ref)


def test_timeout_survives_a_binning_call(orc):
    """A binning call resets its own counters but keeps the timeout count,
    so a timeout met before it is still reported afterwards."""
    api, ctx = api_ctx()
    ctx.synchronize()
    ctx.wait_selftest(10)
    got, ref = _small_bin(api, ctx, orc)
    with pytest.raises(api.UfcError, match="status 4"):
        ctx.synchronize()
    assert np.array_equal(got.cpu().numpy(), ref)
    ctx.synchronize()


def test_selftest_limit_checked():
    api, ctx = api_ctx()
    for bad in (0, -5, (1 << 28) + 1):
        with pytest.raises(api.UfcError, match="status 1"):
            ctx.wait_selftest(bad)
    ctx.synchronize()
