"""Two-rank (gloo, CPU) tests of the multi-process layer: the sum of the
ranks' subvolume count maps equals the single-process map (the map
combination of Sec. 2.4), and gathering per-rank covariance inputs in rank
order reproduces the single-process covariance (Eq. 10)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, tmp):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle
    from paper_1801_05745_gb300 import parallel, synth
    n = 40_000
    x = synth.particles_numpy(n, 2000.0, 5.0, 555)
    chi = np.linspace(150.0, 950.0, 9)
    box = oracle.make_box(2000.0, [1000.0] * 3, n, 0, 8)
    a, b = parallel.shard_range(n, rank, world)
    part, _ = oracle.bin_counts(x[a:b], box, chi, 8)     # this rank's subvolume map
    t = torch.from_numpy(part)
    parallel.allreduce_counts(t)
    full, _ = oracle.bin_counts(x, box, chi, 8)
    ok_counts = bool(np.array_equal(t.numpy(), full))
    # realisation sharding: each rank holds its vectors; gathering them in rank
    # order and taking the covariance equals the single-process covariance
    rng = np.random.default_rng(9)
    v = rng.normal(size=(30, 7))
    mine = torch.from_numpy(v[rank::world].copy())
    gathered = parallel.gather_states(mine)
    allv = np.concatenate([g.numpy() for g in gathered])
    _, cov_all, _ = oracle.covariance(allv, 1)
    _, cov_ref, _ = oracle.covariance(np.concatenate([v[r::world] for r in range(world)]), 1)
    ok_cov = bool(np.allclose(cov_all, cov_ref, rtol=1e-13))
    np.save(os.path.join(tmp, f"r{rank}.npy"), np.array([ok_counts, ok_cov]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_subvolume_sum_and_gather(tmp_path):
    port = _free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        ok = np.load(tmp_path / f"r{r}.npy")
        assert ok.all(), (r, ok)


def test_shard_range_partitions():
    from paper_1801_05745_gb300 import parallel
    for n in (0, 1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            for align in (1, 4):
                spans = [parallel.shard_range(n, r, world, align) for r in range(world)]
                assert spans[0][0] == 0 and spans[-1][1] == n
                assert all(spans[i][1] == spans[i + 1][0] for i in range(world - 1))
                assert all(a % align == 0 for a, _ in spans)


def _welford_worker(rank, world, port, tmp):
    """Realisation sharding through the library (Eq. 10): each rank adds its
    own statistics vectors to its own Welford state with the library's host
    update, the states are gathered in rank order and merged with the
    library's Chan merge (parallel.merge_states on host tensors)."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle
    from paper_1801_05745_gb300 import api, parallel
    d = 9
    rng = np.random.default_rng(21)
    v = rng.normal(size=(47, d)) @ rng.normal(size=(d, d)) + 3.0    # all realisations
    a, b = parallel.shard_range(len(v), rank, world)
    st = np.zeros(1 + d + d * d)
    api.welford_update_host(v[a:b], st)
    states = parallel.gather_states(torch.from_numpy(st))
    merged = parallel.merge_states(None, states, d).numpy()
    n = merged[0]
    mean, M2 = merged[1:1 + d], merged[1 + d:].reshape(d, d)
    m_o, c_o, _ = oracle.covariance(v, 1)
    ok = [n == len(v),
          bool(np.allclose(mean, m_o, rtol=1e-12, atol=1e-12)),
          bool(np.allclose(M2 / (n - 1), c_o, rtol=1e-11, atol=1e-12))]
    # a single state over all vectors in rank order agrees with the merge
    one = np.zeros_like(st)
    api.welford_update_host(v, one)
    ok.append(bool(np.allclose(one, merged, rtol=1e-11, atol=1e-11)))
    np.save(os.path.join(tmp, f"w{rank}.npy"), np.array(ok))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_library_welford_merge(tmp_path):
    port = _free_port()
    mp.spawn(_welford_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        ok = np.load(tmp_path / f"w{r}.npy")
        assert ok.all(), (r, ok)


def _adjoint_worker(rank, world, port, tmp):
    """Subvolume sharding of the map and its gradient (Sec. 2.4) through the
    library's host pieces: each rank bins its shard (oracle), adds its FP64
    partial sum_b A_b n_bp into the all-reduce, forms its share of the
    adjoint sums against the whole map (the definition of
    ufc_kappa_adjoint_sums, in numpy); parallel.allreduce_adjoint_sums
    combines the shares and ufc_kappa_grad_from_sums gives the gradient,
    which must equal the oracle's complex-step gradient of the whole counts.
    Power sums that differ between ranks must raise on every rank."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle
    from paper_1801_05745_gb300 import api, parallel, synth
    n, nside, S = 60_000, 8, 6
    x = synth.particles_numpy(n, 2000.0, 5.0, 777)
    z = np.linspace(0.05, 0.23, S + 1)
    chi = oracle.chi_edges(0.3, 0.7, 0, z)                # Mpc: the gradient in h is not 0
    box_o = oracle.make_box(2000.0, [1000.0] * 3, n, 0, S)
    box_a = api.make_box(2000.0, [1000.0] * 3, n, 0, S)
    a, b = parallel.shard_range(n, rank, world, align=4)
    mine, _ = oracle.bin_counts(x[a:b], box_o, chi, nside)
    full, _ = oracle.bin_counts(x, box_o, chi, nside)
    src = dict(kind=1, z_s=1.5, alpha=2.0, beta=1.5, z0=0.5, z_max=1.5)   # Smail n(z)
    A, B, C, dA, dC = api.kappa_coeffs(api.make_cosmo(0.3, 0.7, 0), [box_a], z, nside,
                                       api.make_source(**src), derivs=True)
    partial = torch.from_numpy(A @ mine.astype(np.float64))
    dist.all_reduce(partial)
    e = partial.numpy() - C                              # the whole map, unrounded
    g = np.random.default_rng(4).normal(size=e.size).astype(np.float32)
    m = mine.astype(np.float64)
    share = np.stack([m @ e, m @ (e * e), m @ g.astype(np.float64), m.sum(1)], axis=1).ravel()
    sums = np.concatenate([share, [e.sum(), (e * e).sum(), (e ** 3).sum(), g.sum(dtype=np.float64)]])
    tot = parallel.allreduce_adjoint_sums(sums, S)
    ok = [bool(np.array_equal(tot[3:4 * S:4], full.sum(1).astype(np.float64)))]
    grad, G, H = api.kappa_grad_from_sums(tot, S, nside, dA, dC, 0.7, 1.3)
    G_or = oracle.kappa_stat_grads(full, nside, 0.3, 0.7, 0, [box_o], z,
                                   oracle.make_source(**src), g)
    want = 0.7 * G_or[0] + 1.3 * G_or[1] + G_or[2]
    sc = 0.7 * np.abs(G_or[0]).max() + 1.3 * np.abs(G_or[1]).max() + np.abs(G_or[2]).max()
    ok.append(bool(np.allclose(grad, want, rtol=1e-9, atol=1e-9 * sc)))
    ok.append(bool(np.all(np.abs(want) > 1e-6 * sc)))   # every parameter's gradient is live
    bad = sums.copy()
    bad[4 * S] += rank * 1e-3 * abs(bad[4 * S])          # rank 1 disagrees on sum_p e_p
    try:
        parallel.allreduce_adjoint_sums(bad, S)
        ok.append(False)
    except RuntimeError:
        ok.append(True)
    np.save(os.path.join(tmp, f"a{rank}.npy"), np.array(ok))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_subvolume_gradient(tmp_path):
    port = _free_port()
    mp.spawn(_adjoint_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        ok = np.load(tmp_path / f"a{r}.npy")
        assert ok.all(), (r, ok)


def _failing_worker(rank, world, port, tmp, mode):
    """Rank 1 fails on the host before the map combination: it raises
    ("raise") or never joins the all-reduce ("absent").  Rank 0 must get an
    error from its collective within the short process-group timeout instead
    of waiting forever."""
    import datetime
    import time
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=3))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_1801_05745_gb300 import parallel
    if rank == 1:
        if mode == "raise":
            raise RuntimeError("rank 1: simulated failure before the all-reduce")
        time.sleep(10)
        os._exit(0)
    t0 = time.monotonic()
    try:
        parallel.allreduce_counts(torch.ones(64, dtype=torch.int32))
        status = 0
    except Exception:
        status = 1
    np.save(os.path.join(tmp, "r0.npy"), np.array([status, time.monotonic() - t0]))
    os._exit(0)


@pytest.mark.parametrize("mode", ["raise", "absent"])
def test_failed_rank_surfaces_as_error(tmp_path, mode):
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, str(tmp_path), mode))
             for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
    alive = [p for p in procs if p.is_alive()]
    for p in alive:
        p.kill()
    assert not alive, "a rank hung past the process-group timeout"
    status, secs = np.load(tmp_path / "r0.npy")
    assert status == 1, "rank 0's all-reduce completed without its peer"
    assert secs < 30
