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
