"""Shared set-up of the GPU parity tests: seeded inputs, the library context
and the oracle's view of the same boxes."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def have_gpu():
    return torch.cuda.is_available()


def api_ctx():
    from paper_1801_05745_gb300 import build
    build.build()
    from paper_1801_05745_gb300 import api
    return api, api.context(0)


def both_boxes(api, orc, L, obs, n_total, lo, hi, R=0):
    return (api.make_box(L, obs, n_total, lo, hi, R), orc.make_box(L, obs, n_total, lo, hi, R))


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()


def boundary_points(orc, nside, n, r_lo, r_hi, seed):
    """Directions on HEALPix pixel edges (equatorial edge lines and cap edge
    curves) at random radii, as FP64 vectors; rounding to FP32 leaves them
    within a few ulp of an edge."""
    rng = np.random.default_rng(seed)
    out = []
    N = nside
    for i in range(n):
        kind = rng.integers(0, 4)
        if kind < 2:   # equatorial edge line N(1/2 + t -+ 3z/4) = k
            z = rng.uniform(-2 / 3, 2 / 3)
            k = rng.integers(0, 5 * N)
            sgn = 1 if kind == 0 else -1
            t = (k / N - 0.5 + sgn * 0.75 * z) % 4.0
        elif kind == 2:   # cap edge N sqrt(3(1-|z|)) t_p = k
            tmpmax = N
            k = rng.integers(1, N)
            tmp = rng.uniform(k + 0.01, tmpmax)
            tp = k / tmp
            za = 1 - (tmp / N) ** 2 / 3
            z = za * (1 if rng.random() < 0.5 else -1)
            t = rng.integers(0, 4) + (tp if rng.random() < 0.5 else 1 - tp)
        else:           # in-ring edge t * ir = k in a cap
            ir = rng.integers(1, N + 1)
            k = rng.integers(0, 4 * ir)
            t = k / ir
            # a height inside ring ir: tmp in (ir - 1, ir)
            tmp = rng.uniform(max(ir - 1, 0) + 0.2, ir - 0.2) if ir > 1 else rng.uniform(0.1, 0.8)
            za = 1 - (tmp / N) ** 2 / 3
            z = za * (1 if rng.random() < 0.5 else -1)
        phi = t * np.pi / 2
        s = np.sqrt(max(0.0, 1 - z * z))
        r = rng.uniform(r_lo, r_hi)
        out.append([r * s * np.cos(phi), r * s * np.sin(phi), r * z])
    return np.array(out)
