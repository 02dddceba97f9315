"""Checkpoint and resume of the covariance over realisations (Sec. 3.2,
Eq. 10-11): a run stopped after some realisations and resumed from its saved
Welford state reaches the uninterrupted state bit for bit; a resumed part
merged afterwards agrees to rounding; the file refuses other runs."""
import os

import numpy as np
import pytest

from paper_1801_05745_gb300 import checkpoint


@pytest.fixture(scope="module")
def api():
    from paper_1801_05745_gb300 import build
    build.build()
    from paper_1801_05745_gb300 import api as a
    return a


def _vectors(d=17, nreal=150):
    rng = np.random.default_rng(12)
    return rng.normal(size=(nreal, d)) @ rng.normal(size=(d, d)) + 2.0


def test_resume_is_bit_identical(api, tmp_path, orc):
    v = _vectors()
    R, d = v.shape
    cfg = {"workload": "test", "nside": 64, "nshell": 12, "seed": 12}
    full = np.zeros(1 + d + d * d)
    api.welford_update_host(v, full)
    st = np.zeros_like(full)
    api.welford_update_host(v[:70], st)
    path = str(tmp_path / "cov.npz")
    checkpoint.save(path, st, d, 70, cfg)
    del st
    st2, nxt = checkpoint.load(path, d, cfg)
    assert nxt == 70
    api.welford_update_host(v[nxt:], st2)
    assert np.array_equal(st2, full)
    # the finished state is the covariance of all realisations (oracle)
    _, cov, _ = orc.covariance(v, 1)
    assert np.allclose(st2[1 + d:].reshape(d, d) / (R - 1), cov, rtol=1e-11, atol=1e-12)
    assert [f for f in os.listdir(tmp_path) if ".tmp" in f] == []


def test_resumed_part_merged(api, tmp_path):
    v = _vectors()
    d = v.shape[1]
    full = np.zeros(1 + d + d * d)
    api.welford_update_host(v, full)
    a = np.zeros_like(full)
    api.welford_update_host(v[:64], a)
    checkpoint.save(str(tmp_path / "a.npz"), a, d, 64)
    b = np.zeros_like(full)                      # the rest, in a state of its own
    api.welford_update_host(v[64:], b)
    a2, _ = checkpoint.load(str(tmp_path / "a.npz"), d)
    api.welford_merge_host(a2, b, d)
    assert a2[0] == full[0]
    assert np.allclose(a2, full, rtol=1e-12, atol=1e-12 * np.abs(full).max())


def test_checkpoint_refuses_other_runs(tmp_path):
    d = 3
    st = np.zeros(1 + d + d * d)
    st[0] = 2.0
    path = str(tmp_path / "c.npz")
    checkpoint.save(path, st, d, 2, {"nside": 64})
    checkpoint.save(path, st, d, 2, {"nside": 64})          # overwrite in place
    with pytest.raises(ValueError):
        checkpoint.load(path, d, {"nside": 128})
    with pytest.raises(ValueError):
        checkpoint.load(path, d + 1)
    with pytest.raises(ValueError):
        checkpoint.save(path, st[:-1], d, 2)
    with pytest.raises(ValueError):
        checkpoint.save(path, st, d, 1)                     # fewer than the state's n
    with pytest.raises(TypeError):
        checkpoint.save(path, st.astype(np.float32), d, 2)
    other = str(tmp_path / "o.npz")
    np.savez(other, format=np.array("something else"), d=np.int64(d))
    with pytest.raises(ValueError):
        checkpoint.load(other, d)
    got, nxt = checkpoint.load(path, d, {"nside": 64})
    assert nxt == 2 and np.array_equal(got, st)
