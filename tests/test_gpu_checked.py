"""Index tests of the checked build (-DUFC_CHECKED): the report path
(ufc_check_selftest, in every build) and a run of the binning paths and the
batched kernel on the checked library, which must find no failed test and
give the oracle's counts."""
import os
import subprocess
import sys

import numpy as np
import pytest

from tests.gpu_common import api_ctx

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_failed_index_test_is_reported_once():
    api, ctx = api_ctx()
    ctx.check_selftest(3, 5)                     # in bounds: nothing recorded
    ctx.synchronize()
    ctx.check_selftest(10, 5)
    ctx.check_selftest(-1, 5)
    with pytest.raises(api.UfcError, match=r"2 index test\(s\) failed.*site 0: index 10, bound 5"):
        ctx.synchronize()
    ctx.synchronize()                            # the report cleared the record
    # the context stays usable
    x = torch.zeros(4, device="cuda")
    assert float((x + 1).sum()) == 4.0


_SCRIPT = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
import oracle
from paper_1801_05745_gb300 import api, synth
assert api.CHECKED and api.LIB_PATH.endswith("_checked.so")
ctx = api.context(0)
n = 600_000
x1 = synth.particles_numpy(n, 2000.0, 5.0, 41)
x2 = synth.particles_numpy(n, 6400.0, 20.0, 42)
z = np.linspace(0.1, 1.5, 41)
chi = oracle.chi_edges(0.3, 0.7, 1, z)
split = int(np.argmin(np.abs(chi - 1000.0)))
ba = [api.make_box(2000.0, [1000.0] * 3, n, 0, split), api.make_box(6400.0, [3200.0] * 3, n, split, 40)]
bo = [oracle.make_box(2000.0, [1000.0] * 3, n, 0, split), oracle.make_box(6400.0, [3200.0] * 3, n, split, 40)]
xs = [torch.from_numpy(x1).cuda(), torch.from_numpy(x2).cuda()]
ref = oracle.bin_counts(x1, bo[0], chi, 256)[0].astype(np.int64) + oracle.bin_counts(x2, bo[1], chi, 256)[0]
for path in ("dense", "direct"):
    c = ctx.bin(xs, ba, chi, 256, path=path)
    ctx.synchronize()                            # raises if an index test failed
    assert np.array_equal(c.cpu().numpy(), ref), path
# the batched kernel (small maps): 3 realisations
src = api.make_source(kind=1, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5)
A, B, C = api.kappa_coeffs(api.make_cosmo(), ba, z, 64, src)
st = api.welford_state(6 + 20)
ctx.batched_stats([xs] * 3, [ba] * 3, chi, 64, np.array([A] * 3), np.array([C] * 3),
                  -0.05, 0.2, 20, st)
ctx.synchronize()
print("CHECKED-OK")
"""


def test_checked_build_runs_clean():
    from paper_1801_05745_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, UFC_CHECKED="1")
    r = subprocess.run([sys.executable, "-c", _SCRIPT, ROOT], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0 and "CHECKED-OK" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]


def test_binning_suites_on_checked_build():
    """The binning, key and snapshot test files run on the checked library;
    every test ends with a synchronize that would report a failed index test
    (tests/conftest.py)."""
    from paper_1801_05745_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, UFC_CHECKED="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu",
                        "-p", "no:cacheprovider", "tests/test_gpu_bin.py",
                        "tests/test_gpu_keys.py", "tests/test_gpu_snapshot.py"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
