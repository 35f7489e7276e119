"""Multi-GPU host logic on CPU with gloo (world size 2): each rank propagates its own batch
(weak scaling, no data-path collective); the benchmark takes the slowest rank's time and
the sum of the steps; per-rank batches are disjoint and seeded apart."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    from paper_1410_5323_gb300 import inputs as I

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, acc, att = bench.aggregate(dist, 100.0 + 50.0 * rank, 1000 * (rank + 1), 1500 * (rank + 1),
                                   torch.device("cpu"))
    w = I.workload("fp64_64cube_1k_protons")
    parts = I.make_particles(64, w.particle_seed + 7919 * rank, w.species, w.energy, uid_offset=rank * 64)
    uids = torch.from_numpy(parts.u[:, 0].copy())
    gathered = [torch.zeros_like(uids) for _ in range(world)]
    dist.all_gather(gathered, uids)
    out[rank] = (ms, acc, att, parts.uid.tolist(), [g.tolist() for g in gathered])
    dist.destroy_process_group()


def test_two_rank_aggregation_and_sharding():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29500 + os.getpid() % 2000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        ms, acc, att, uids, gathered = out[r]
        assert ms == 150.0                     # slowest rank
        assert acc == 3000.0 and att == 4500.0  # steps summed over ranks
    u0, u1 = set(out[0][3]), set(out[1][3])
    assert not (u0 & u1) and u0 | u1 == set(range(128))     # disjoint uids
    g = out[0][4]
    assert not np.allclose(g[0], g[1])                     # batches seeded apart


def _run_ranks(target, world, *extra):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = 29500 + (os.getpid() * 7 + world) % 2000
    procs = [ctx.Process(target=target, args=(r, world, port, out) + extra) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    return dict(out)


def _grid_shard_worker(rank, world, port, out, n_grids, grid_n, per_grid, dmax):
    """One rank of the batching form split by grid id: builds only its realisations, runs the
    oracle on their particles, hands its records to rank 0 (all_gather_object)."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import oracle as O
    from paper_1410_5323_gb300 import inputs as I
    from paper_1410_5323_gb300 import shard

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = I.workload("batched_64x128cube_12.8M_protons")
    ids = shard.grid_shard(n_grids, rank, world)
    grids, _ = I.batched_grids(w, n_grids=n_grids, grid_n=grid_n, ids=ids)
    parts = shard.take_grid_shard(I.batched_particles(w, per_grid, n_grids=n_grids), ids)
    st = O.OracleState(len(parts))
    O.inject(st, parts, 1)
    rc, _ = O.propagate(st, [O.OracleField(g, w.spacing_m) for g in grids], None, w.tol, w.hmin_m,
                        w.hmax_m, dmax, seed=1)
    snap = st.snapshot()
    snap["grid_id"] = ids[snap["grid_id"]]          # back to global realisation ids
    got = [None] * world
    dist.all_gather_object(got, (rc, len(grids), snap))
    if rank == 0:
        out["gathered"] = got
    dist.destroy_process_group()


def test_two_rank_grid_shards_equal_the_single_run_bit_for_bit():
    """The batching form split by grid id over two gloo ranks (each holds 3 of 6 realisations
    and their particles, runs the FP64 oracle on them): the union of the two ranks' records
    equals one process running all six realisations, bit for bit in every column."""
    pytest.importorskip("torch")
    import oracle as O
    from paper_1410_5323_gb300 import inputs as I
    from _parity import by_uid

    n_grids, grid_n, per_grid, dmax = 6, 16, 5, 4 * I.MPC
    out = _run_ranks(_grid_shard_worker, 2, n_grids, grid_n, per_grid, dmax)
    got = out["gathered"]
    assert [g[0] for g in got] == [0, 0] and [g[1] for g in got] == [3, 3]
    union = {k: np.concatenate([g[2][k] for g in got]) for k in got[0][2]}
    w = I.workload("batched_64x128cube_12.8M_protons")
    grids, _ = I.batched_grids(w, n_grids=n_grids, grid_n=grid_n)
    parts = I.batched_particles(w, per_grid, n_grids=n_grids)
    st = O.OracleState(len(parts))
    O.inject(st, parts, 1)
    rc, _ = O.propagate(st, [O.OracleField(g, w.spacing_m) for g in grids], None, w.tol, w.hmin_m,
                        w.hmax_m, dmax, seed=1)
    assert rc == 0
    a, b = by_uid(st.snapshot()), by_uid(union)
    assert len(a["uid"]) == len(b["uid"]) == n_grids * per_grid
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def _adjoint_worker(rank, world, port, out, n, grid_n, n_steps):
    """One rank of the differentiation form: its block of chains through the oracle's
    recorded forward and reverse pass, its share of dL/dB summed over ranks by all-reduce."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_1410_5323_gb300 import shard

    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from paper_1410_5323_gb300 import inputs as I

    g, y0, kap, lam = _adjoint_case(n, grid_n)
    of = O.OracleField(g, 0.25 * I.MPC)
    lo, hi = shard.block_range(n, rank, world)
    gb = np.zeros(g.shape)
    yb = {}
    for i in range(lo, hi):
        h, _ = O.record_steps(of, kap[i], y0[i], 1e-4, I.KPC, I.MPC, n_steps)
        yb[i] = O.adjoint(of, kap[i], y0[i], h, lam[i], gb)[0]
    t = torch.from_numpy(gb)
    shard.allreduce_sum_(t, dist)
    got = [None] * world
    dist.all_gather_object(got, yb)
    if rank == 0:
        out["grid_bar"] = t.numpy().copy()
        out["y0_bar"] = {k: v for d in got for k, v in d.items()}
    dist.destroy_process_group()


def _adjoint_case(n, grid_n):
    from paper_1410_5323_gb300 import inputs as I

    g = I.kolmogorov_grid(grid_n, 0.25 * I.MPC, 2, grid_n // 2, 1e-13, 5).astype(np.float32)
    p = I.make_particles(n, 15, energy=("fixed", 10 ** 19.5))
    y0 = np.concatenate([p.x, p.u], axis=1)
    kap = (p.Z.astype(np.float64) * 299792458.0) / p.E
    rng = np.random.default_rng(2)
    lam = np.concatenate([np.zeros((n, 3)), rng.standard_normal((n, 3))], axis=1)
    return g, y0, kap, lam


def test_two_rank_adjoint_gradient_is_summed_by_allreduce():
    """The differentiation form over two gloo ranks: each rank's chains give the same per-chain
    gradients as one process (bit for bit), and the all-reduced grid gradient equals the
    single-process accumulation up to the order of the additions."""
    pytest.importorskip("torch")
    import oracle as O
    from paper_1410_5323_gb300 import inputs as I

    n, grid_n, n_steps = 10, 16, 60
    out = _run_ranks(_adjoint_worker, 2, n, grid_n, n_steps)
    g, y0, kap, lam = _adjoint_case(n, grid_n)
    of = O.OracleField(g, 0.25 * I.MPC)
    gb = np.zeros(g.shape)
    for i in range(n):
        h, _ = O.record_steps(of, kap[i], y0[i], 1e-4, I.KPC, I.MPC, n_steps)
        yb, _ = O.adjoint(of, kap[i], y0[i], h, lam[i], gb)
        assert np.array_equal(yb, out["y0_bar"][i]), i
    got = out["grid_bar"]
    assert np.array_equal(got != 0, gb != 0) and np.count_nonzero(gb) > 0
    assert np.allclose(got, gb, rtol=1e-12, atol=1e-15 * np.abs(gb).max())


def test_block_and_grid_partitions():
    from paper_1410_5323_gb300 import inputs as I
    from paper_1410_5323_gb300 import shard

    for n, world in ((10, 3), (64, 8), (5, 8), (0, 2)):
        r = [shard.block_range(n, k, world) for k in range(world)]
        assert r[0][0] == 0 and r[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        assert max(h - l for l, h in r) - min(h - l for l, h in r) <= 1
    w = I.workload("batched_64x128cube_12.8M_protons")
    p = I.batched_particles(w, 3, n_grids=5)
    parts = [shard.take_grid_shard(p, shard.grid_shard(5, k, 2)) for k in range(2)]
    assert sorted(np.concatenate([q.uid for q in parts]).tolist()) == p.uid.tolist()
    assert parts[0].grid_id.tolist() == [0, 0, 0, 1, 1, 1, 2, 2, 2]
    assert parts[1].grid_id.tolist() == [0, 0, 0, 1, 1, 1]
    with pytest.raises(ValueError):
        shard.block_range(4, 2, 2)
