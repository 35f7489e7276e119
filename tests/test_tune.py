"""Autotuner search logic and cache (host only), and one tuning run on the GPU."""
import json

import numpy as np
import pytest

from paper_1410_5323_gb300 import inputs as I
from paper_1410_5323_gb300 import tune


def test_coordinate_descent_finds_separable_optimum():
    target = {"block_size": 256, "blocks_per_sm": 1, "cadence": 4, "order": 3, "slice_steps": 4000}

    def measure(cfg):
        return 100.0 - sum(abs(tune.SPACE[k].index(cfg[k]) - tune.SPACE[k].index(target[k]))
                           for k in target)

    best, val, log = tune.coordinate_descent(measure, passes=3)
    assert best == target and val == 100.0
    assert len(log) > 5


def test_coordinate_descent_skips_failing_configs():
    def measure(cfg):
        return None if cfg["block_size"] == 256 else float(cfg["cadence"])

    best, val, _ = tune.coordinate_descent(measure)
    assert best["block_size"] != 256 and best["cadence"] == 4


def test_cache_roundtrip(tmp_path):
    path = str(tmp_path / "c.json")
    tune.store_cache("k1", {"config": {"a": 1}}, path)
    tune.store_cache("k2", {"config": {"a": 2}}, path)
    data = json.load(open(path))
    assert data["k1"]["config"] == {"a": 1} and data["k2"]["config"] == {"a": 2}
    assert tune.load_cache(str(tmp_path / "missing.json")) == {}


def test_signature_distinguishes_workloads():
    a = tune.signature(1, 1000, (128, 128, 128), 64, False)
    b = tune.signature(1, 1000, (128, 128, 128), 1, False)
    assert a != b


@pytest.mark.gpu
def test_autotune_on_gpu_returns_a_valid_config(tmp_path):
    import paper_1410_5323_gb300 as crp

    grids = [I.kolmogorov_grid(32, 0.25 * I.MPC, 2, 16, b, s).astype(np.float32)
             for s, b in ((1, 1e-13), (2, 1e-12))]
    p = I.make_particles(4000, 3, energy=("loguniform", 1e18, 1e20))
    p.grid_id[:] = np.arange(4000) % 2
    sim = crp.Simulation([crp.Field(g, 0.25 * I.MPC) for g in grids], None, capacity=4000)
    space = {"block_size": [64, 128], "cadence": [1, 2], "order": [2, 3], "slice_steps": [0, 500],
             "blocks_per_sm": [0]}
    cfg = tune.autotune(sim, lambda: sim.inject(p), crp.FORM_MIXED, 1e-4, I.KPC, I.MPC, 20 * I.MPC,
                        "test", use_cache=False, space=space, cache_path=str(tmp_path / "t.json"))
    assert cfg["block_size"] in (64, 128) and cfg["order"] in (2, 3)
    assert "test" in next(iter(json.load(open(tmp_path / "t.json"))))
