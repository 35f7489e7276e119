"""Autotuner for the propagate launch: block size, blocks per SM, refill cadence, work-list
order and slice budget (max_steps per slice of the graph loop), chosen by measured
throughput on a sample of the workload and cached per (GPU, form, workload signature).

The search is coordinate descent from the library defaults: each parameter in turn is
swept with the others fixed, the best value kept, and the pass repeated while it improves.
Measurements run the real propagation through the C ABI; nothing here computes physics.
"""
from __future__ import annotations

import json
import os
import time

SPACE = {
    "block_size": [64, 128, 256],
    "blocks_per_sm": [0, 1, 2],          # 0: occupancy limit
    "cadence": [1, 2, 4],
    "order": [2, 3, 1],                  # cost, grid-major, slot
    "slice_steps": [0, 4000, 16000],     # 0: one propagate call; else graph loop slices
}
DEFAULT = {"block_size": 128, "blocks_per_sm": 0, "cadence": 1, "order": 2, "slice_steps": 0}

CACHE = os.environ.get("CRP_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache",
                                                      "crp_tune.json"))


def coordinate_descent(measure, space=None, start=None, passes: int = 2):
    """measure(config) -> throughput (higher is better), or None for an invalid config.
    Returns (best_config, best_value, log)."""
    space = space or SPACE
    best = dict(start or DEFAULT)
    best_v = measure(best)
    log = [(dict(best), best_v)]
    if best_v is None:
        raise RuntimeError("the starting configuration failed")
    for _ in range(passes):
        improved = False
        for key, values in space.items():
            for v in values:
                if v == best[key]:
                    continue
                cand = dict(best)
                cand[key] = v
                val = measure(cand)
                log.append((dict(cand), val))
                if val is not None and val > best_v * 1.01:
                    best, best_v, improved = cand, val, True
        if not improved:
            break
    return best, best_v, log


def signature(form: int, n_particles: int, grid_shape, n_fields: int, tables: bool) -> str:
    return f"form{form}-n{n_particles}-g{'x'.join(map(str, grid_shape))}-f{n_fields}-t{int(tables)}"


def _gpu_name() -> str:
    try:
        import torch

        return torch.cuda.get_device_name(0)
    except Exception:   # noqa: BLE001 - name only labels the cache entry
        return "unknown"


def load_cache(path: str = CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store_cache(key: str, entry: dict, path: str = CACHE) -> None:
    data = load_cache(path)
    data[key] = entry
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def run_config(sim, inject, cfg: dict, form: int, tol: float, hmin: float, hmax: float,
               dmax: float, max_slices: int = 1 << 16):
    """Propagate one injected sample with cfg; returns (accepted steps/s, seconds, rc)."""
    import torch

    sim.reset()
    inject()
    torch.cuda.synchronize()
    kw = dict(form=form, block_size=cfg["block_size"], blocks_per_sm=cfg["blocks_per_sm"],
              cadence=cfg["cadence"], order=cfg["order"])
    t0 = time.perf_counter()
    if cfg["slice_steps"] > 0:
        sim.propagate_loop(tol, hmin, hmax, dmax, max_steps=cfg["slice_steps"],
                           max_slices=max_slices, **kw)
    else:
        sim.propagate(tol, hmin, hmax, dmax, **kw)
    rc = sim.sync(0.0, raise_on_error=False)
    dt = time.perf_counter() - t0
    c = sim.counts()
    if rc != 0 or c["n_active"] != 0:
        return None, dt, rc
    return c["accepted"] / dt, dt, rc


def autotune(sim, inject, form: int, tol: float, hmin: float, hmax: float, dmax: float,
             sig: str, use_cache: bool = True, passes: int = 1, space=None, cache_path: str = CACHE):
    """Tune on the sample that `inject()` puts into `sim`; returns the best config dict."""
    key = f"{_gpu_name()}|{sig}"
    if use_cache:
        hit = load_cache(cache_path).get(key)
        if hit:
            return hit["config"]

    def measure(cfg):
        v, _, _ = run_config(sim, inject, cfg, form, tol, hmin, hmax, dmax)
        return v

    best, best_v, log = coordinate_descent(measure, space=space, passes=passes)
    store_cache(key, {"config": best, "steps_per_s": best_v,
                      "log": [[c, v] for c, v in log]}, cache_path)
    return best
