#!/usr/bin/env python
"""Benchmark: particle RK-steps/s of the 3D propagation hot path (arXiv:1410.5323, CRPropa 3).

Workload (default): 10^6 nuclei (H/He-4/N-14/Fe-56 = 0.4/0.3/0.2/0.1, E^-2 on
[1e18, 10^20.5] eV, isotropic from the origin) through a 256^3 FP32 Kolmogorov grid
(0.25 Mpc cells, l = 2-32 cells, B_rms = 1 nG) with synthetic loss / photo-disintegration
tables, to 500 Mpc, FP64 form. One bench step = the whole hot path over that batch:
inject (device-resident columns) + propagate every primary and every secondary to the
distance limit. value = accepted RK steps of all particles / device time.

Prints one JSON line (rank 0). Synthetic seeded inputs; no datasets.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1410_5323_gb300 import inputs as I  # noqa: E402
from paper_1410_5323_gb300 import shard  # noqa: E402

METRIC = "particle RK-steps/s (accepted Cash-Karp steps summed over particles / propagate time)"
UNIT = "steps/s"

# Algorithmic FP64 work of the method (counted from its formulas; each +,-,*,/,sqrt,max one
# flop, each elementary function one flop):
#   per attempt: 5 field evaluations (stages 2-6) x (lookup 69 + Lorentz 12) = 405, stage
#   sums 210, 5th-order update 54, error estimate 60, squared error norms 10 + (h tol)^2 2,
#   h x step factor and its clamp 2 (the factor itself is FP32 work)  -> 743
#   per accepted step: the next step's first field evaluation 81 (rejected attempts reuse
#   it), kappa = Z c / E 2 -> 83; with tables (the rates themselves are FP32 work, below):
#   distance bid 1, max(tau, 0) 1, three bid comparisons 3, loss h R, exp, E x 3, tau - h R 2
#   -> 10 more
FLOP_PER_ATTEMPT = 743
FLOP_PER_ACCEPTED = 83
FLOP_PER_ACCEPTED_TABLES = 10
# FP64 pipe of one GB300: 2 FP64 lanes/clk/SM x 152 SMs x 2070 MHz = 6.29e11 ops/s,
# 1.259e12 FLOP/s counting an FMA as two (the FP64 form issues no FMA: ceiling 0.5).
FP64_PEAK_TFLOPS = 152 * 2 * 2.070e9 * 2 / 1e12
FP64_OPS_PEAK_T = 152 * 2 * 2.070e9 / 1e12          # FP64 pipe instructions (T ops/s)
FP32_PEAK_TFLOPS = 152 * 128 * 2.070e9 * 2 / 1e12   # FFMA lanes x 2
# Mixed form: FP64 ops that remain per attempt: none outside the accept decision's guard band
# (the FP32 norms certify the FP64 decision there; inside it, a fraction of order 1e-5 of the
# attempts, 2 x (mul + 2 fma), max, compare); per accepted step (path length add, distance
# bid and its conversion, compare, loss factor) 5; the FP32 flops per attempt (6 x (lookup 60
# + Lorentz 9) + stages 120 + update/error 66 + squared norms and ratio 12, band tests 3).
MIXED_FP64_OPS_PER_ATTEMPT = 0
MIXED_FP64_OPS_PER_ACCEPTED = 5
MIXED_FP32_FLOP_PER_ATTEMPT = 615
# DRAM bytes (read + write) of one lens launch measured by ncu on the current kernels, keyed by
# the number of maps (the lens summary under profiles/ names the command).
LENS_DRAM_BYTES = {1: 2.406e8, 32: 5.531e8}
# Modulated fields add one scalar trilinear lookup per field evaluation: FP64 form 42 each
# (axes 12, weights 12, 8 products, 7 sums, 3 products m*B), 5 x 42 = 210 per attempt and 42
# per accepted step; mixed form
# 6 x 38 FP32 flops per attempt and, per accepted step, the step-start modulation cell in
# FP64 (3 x (2 widenings, 3 add, 1 mul, floor, 2 conversions, 1 mul)) = 33 FP64 ops.
MOD_FLOP_PER_ATTEMPT = 210
MOD_FLOP_PER_ACCEPTED = 42
MIXED_MOD_FP64_OPS_PER_ACCEPTED = 33
MIXED_MOD_FP32_FLOP_PER_ATTEMPT = 228
# DRAM bytes (read + write) per attempted step of the propagate kernels, measured by ncu at
# reduced batch (both launches of one call; the summaries under profiles/ name the command);
# traffic of a call = this x its attempts. Keyed by (workload, form).
DRAM_BYTES_PER_ATTEMPT = {("fp64_256cube_1M_nuclei", "fp64"): 139.1,
                          ("fp64_256cube_1M_nuclei", "mixed"): 99.3,      # cell-major grid copy
                          ("modulated_440cube_300kpc_x_256cube_50kpc_1M_nuclei", "fp64"): 372.8}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--form", default=None, choices=["fp64", "mixed"],
                    help="form whose throughput is `value` (default: fp64 for the FP64 workload, "
                         "mixed for the precision and batching workloads); the other form is "
                         "reported under `forms` for the FP64 workload")
    ap.add_argument("--no-other-form", action="store_true")
    ap.add_argument("--workload", default="fp64_256cube_1M_nuclei")
    ap.add_argument("--n-particles", type=int, default=0, help="override batch size (testing)")
    ap.add_argument("--grid-n", type=int, default=0, help="override grid size (profiling)")
    ap.add_argument("--bf16", action="store_true", help="store the grid as BF16 + scale (profiling)")
    ap.add_argument("--cpu-sample", type=int, default=16384, help="primaries in the oracle sample")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--block-size", type=int, default=0)
    ap.add_argument("--cadence", type=int, default=0)
    ap.add_argument("--order", type=int, default=0, help="work-list order (CRP_ORDER_*); 0: default")
    ap.add_argument("--n-maps", type=int, default=1, help="lens workload: maps per rigidity bin")
    ap.add_argument("--lens-group", type=int, default=0, help="lens workload: lanes per row for one map; 0: default")
    ap.add_argument("--e2e-steps", type=int, default=5, help="steps of the end-to-end measurement (at most --steps)")
    ap.add_argument("--no-forms", action="store_true",
                    help="default workload only: skip the precision (1024^3 BF16), batching and adjoint legs")
    ap.add_argument("--forms-steps", type=int, default=2, help="timed steps of each extra leg")
    ap.add_argument("--forms-warmup", type=int, default=3, help="warm-up steps of each extra leg")
    ap.add_argument("--slice-steps", type=int, default=-1,
                    help="> 0: graph loop of slices of this many steps; 0: one call; -1: workload default")
    return ap.parse_args()


# ---------------------------------------------------------------------------------------
def workload_for(args) -> I.Workload:
    w = I.workload(args.workload)
    if args.grid_n:
        w.grid_n = args.grid_n
        w.name = f"{w.name} (grid {args.grid_n}^3)"
    if args.bf16:
        w.bf16 = True
        w.name = f"{w.name} (bf16 grid)"
    return w


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class GridInput:
    """One field grid in the form both sides need: the library's Field and the oracle's."""

    def __init__(self, grid=None, bf16=None, scale=1.0, mod=None, mod_spacing=1.0):
        self.grid, self.bf16, self.scale = grid, bf16, scale
        self.mod, self.mod_spacing = mod, mod_spacing

    def field(self, crp, spacing):
        if self.bf16 is not None:
            f = crp.Field(self.bf16, spacing, scale=self.scale)
        else:
            f = crp.Field(self.grid, spacing)
        if self.mod is not None:
            f.modulate(self.mod, self.mod_spacing)
        return f

    def oracle_field(self, O, spacing):
        mkw = dict(modulation=self.mod, mod_spacing=self.mod_spacing)
        if self.bf16 is not None:
            import torch

            bits = self.bf16.view(torch.int16).cpu().numpy().view(np.uint16)
            return O.OracleField(bits, spacing, scale=self.scale, dtype=O.BF16, **mkw)
        return O.OracleField(self.grid, spacing, **mkw)


def build_inputs(w: I.Workload, n: int, rank: int):
    """Field grids (list of GridInput), tables, particles of the workload (this rank's batch)."""
    tables = I.synthetic_tables() if w.interactions else None
    if w.bf16:              # generated and quantised on the device (BF16 + one FP32 scale)
        import torch

        B = I.kolmogorov_grid_torch(w.grid_n, w.lmin_cells, w.lmax_cells, w.brms_t, w.grid_seed)
        q, scale = I.quantize_bf16(B)
        del B
        torch.cuda.empty_cache()       # the FFT's working memory goes back to the device
        parts = I.make_particles(n, w.particle_seed + 7919 * rank, w.species, w.energy,
                                 uid_offset=rank * n)
        return [GridInput(bf16=q, scale=scale)], tables, parts
    if w.n_grids > 1:           # realisations split by grid id over the ranks (one job)
        ws = dist_env()[0]
        ids = shard.grid_shard(w.n_grids, rank, ws)
        grids, _ = I.batched_grids(w, ids=ids)
        per = max(1, n // w.n_grids)
        parts = shard.take_grid_shard(I.batched_particles(w, per, seed=w.particle_seed), ids)
        return [GridInput(grid=g) for g in grids], tables, parts
    grid = I.kolmogorov_grid(w.grid_n, w.spacing_m, w.lmin_cells, w.lmax_cells, w.brms_t,
                             w.grid_seed).astype(np.float32)
    if w.spectrum is not None:     # species, energies, directions are drawn on the device
        parts = I.make_particles(n, w.particle_seed + 7919 * rank, (("H", 1.0),), ("fixed", 1e19),
                                 uid_offset=rank * n)
    else:
        parts = I.make_particles(n, w.particle_seed + 7919 * rank, w.species, w.energy,
                                 uid_offset=rank * n)
    if w.mod_n:             # modulated field; sources follow the matter density
        rho = I.density_field(w.mod_n, w.mod_lmin_cells, w.mod_lmax_cells, w.mod_sigma_ln, w.mod_seed)
        mod = I.modulation_from_density(rho)
        parts.x[:] = I.density_positions(n, rho, w.mod_spacing_m, w.particle_seed + 7919 * rank)
        del rho
        return [GridInput(grid=grid, mod=mod, mod_spacing=w.mod_spacing_m)], tables, parts
    return [GridInput(grid=grid)], tables, parts


def oracle_sample_index(w: I.Workload, n_total: int, sample: int) -> np.ndarray:
    """Primaries the oracle reruns: the first ones, or the first of every realisation."""
    if w.n_grids > 1:
        per_grid = n_total // w.n_grids
        k = max(1, min(per_grid, sample // w.n_grids))
        return (np.arange(w.n_grids)[:, None] * per_grid + np.arange(k)[None, :]).ravel()
    return np.arange(min(sample, n_total))


def oracle_sources(w: I.Workload, parts, lo: int, count: int, seed: int):
    """For Eq. 1 workloads: primaries lo .. lo+count-1 as the device draws them (the oracle's
    sampler, same Philox counters), at the batch's positions; else the batch's own."""
    sub = parts.take(np.arange(lo, lo + count))
    if w.spectrum is None:
        return sub
    import oracle as O

    species, alpha, rcut, emin, emax = w.spectrum
    A, Z, E, u, _ = O.source_sample(O.spectrum(species, alpha, rcut, emin, emax), seed,
                                    int(parts.uid[lo]), count)
    sub.A[:], sub.Z[:], sub.E[:], sub.u[:] = A, Z, E, u
    return sub


def capacity_hint(w: I.Workload, parts) -> int:
    if w.spectrum is not None:       # every primary may be Fe-56: room for 55 nucleons each
        return int(len(parts) * max(a for a, _, _ in w.spectrum[0]))
    return capacity_for(parts)


def aggregate(dist, total_ms: float, accepted: float, attempted: float, device):
    """Whole-job figures over ranks: the slowest rank's time, the sum of the steps."""
    if dist is None:
        return float(total_ms), float(accepted), float(attempted)
    import torch

    t = torch.tensor([total_ms, accepted, attempted], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(t[1]), float(t[2])


def capacity_for(parts) -> int:
    return int(len(parts) + np.sum(parts.A.astype(np.int64) - 1))


class ClockSampler:
    """nvidia-smi sampling (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(w, grids, tables, parts, sample: int, form_desc: str):
    """The oracle, as it stands, on a bounded sample of the same workload."""
    import oracle as O

    idx = oracle_sample_index(w, len(parts), sample)
    sub = oracle_sources(w, parts, 0, len(idx), w.rng_seed) if w.spectrum is not None else parts.take(idx)
    cap = capacity_for(sub)
    st = O.OracleState(cap)
    ot = O.OracleTables(tables) if tables is not None else None
    O.inject(st, sub, w.rng_seed, ot)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    rc, stats = O.propagate(st, [g.oracle_field(O, w.spacing_m) for g in grids], ot, w.tol,
                            w.hmin_m, w.hmax_m, w.dmax_m, seed=w.rng_seed, n_threads=threads,
                            box=I.workload_box(w))
    dt = time.perf_counter() - t0
    return ({"value": stats["accepted"] / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
             "per_core": stats["accepted"] / dt / threads,
             "sample": f"{len(sub)} primaries of the same batch (+{stats['secondaries']} "
                       f"secondaries), full {w.dmax_m / I.MPC:.0f} Mpc, {stats['accepted']} "
                       f"accepted steps in {dt:.2f} s ({form_desc} oracle)",
             "rc": rc}, st.snapshot())


def traffic_for(workload, form, attempted, calls):
    """DRAM bytes per propagate call (both launches), from the measured bytes per attempt."""
    key = (workload, form)
    if key not in DRAM_BYTES_PER_ATTEMPT or calls <= 0:
        return None
    return DRAM_BYTES_PER_ATTEMPT[key] * attempted / calls


# Gathered bytes of one trilinear lookup: 8 corners x 3 components of the stored value type
# (algorithmic: the fourth lane of a node vector and the cell-major copy's duplication are
# not counted); a modulated field adds 8 FP32 modulation corners. The FP64 form evaluates the
# field 5 times per attempt and once per accepted step (the next step's k1, reused by
# rejected attempts) and reads FP64 values (its widened copy); the precision form 6 times
# per attempt, reading FP32 or BF16 values.
LOOKUP_BYTES = {"f64": 8 * 3 * 8, "f32": 8 * 3 * 4, "bf16": 8 * 3 * 2}
MOD_LOOKUP_BYTES = 8 * 4
# FP32 work of the FP64 form: the step-size factor per attempt (log2 of three FP64 values
# from their bits, 3 x 14, their combination 6, the clamped power 26); with tables, per
# accepted step the rates (two bit-level log2 28, coordinate 8, two interpolated powers of
# two 2 x 27) and the two bid quotients 2.
FP64_FORM_FP32_FLOP_PER_ATTEMPT = 74
FP64_FORM_FP32_FLOP_PER_ACCEPTED_TABLES = 92
L2_BYTES = 126 * 1024 * 1024


def measured_peaks() -> dict:
    """HBM copy bandwidth measured on this machine's GPUs (GB/s), else the stated fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return {"hbm_gbs": float(json.load(open(path))["hbm_gbs"]),
                "hbm_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    return {"hbm_gbs": 6800.0, "hbm_source": "fallback 6.8 TB/s (of fallback)"}


def measure_l2_gbs(dev) -> float:
    """Copy bandwidth of a 2 x 24 MiB working set (read + write bytes) that stays in L2,
    best of 20 CUDA-event timed repetitions of 10 copies."""
    import torch

    a = torch.ones(24 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    b = torch.empty_like(a)
    for _ in range(20):
        b.copy_(a)
    best = float("inf")
    for _ in range(20):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            b.copy_(a)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    return 10 * 2 * a.numel() * 4 / best / 1e9


def roofline_terms(form, attempted, accepted, tables, prop_s, modulated=False, grid_dtype="f32",
                   grid_bytes=0, peaks=None):
    """The three terms of the roofline of one propagate form (each against its own peak):
    gathered bytes of the lookups at HBM (or L2, when the grid the form reads fits in L2),
    FP32 FLOPs at the FP32 peak, FP64 FLOPs (FP64 form) or FP64 pipe ops (precision form) at
    the FP64 peak. Returns {name: term}."""
    peaks = peaks or measured_peaks()
    in_l2 = 0 < grid_bytes <= L2_BYTES and peaks.get("l2_gbs")
    if form == "fp64":
        lookups = 5 * attempted + accepted
        gbytes = lookups * (LOOKUP_BYTES["f64"] + (MOD_LOOKUP_BYTES if modulated else 0))
        per_att = FLOP_PER_ATTEMPT + (MOD_FLOP_PER_ATTEMPT if modulated else 0)
        per_acc = (FLOP_PER_ACCEPTED + (MOD_FLOP_PER_ACCEPTED if modulated else 0)
                   + (FLOP_PER_ACCEPTED_TABLES if tables else 0))
        f64 = per_att * attempted + per_acc * accepted
        f32 = FP64_FORM_FP32_FLOP_PER_ATTEMPT * attempted + (FP64_FORM_FP32_FLOP_PER_ACCEPTED_TABLES * accepted
                                                              if tables else 0)
        t64 = {"achieved": f64 / prop_s / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
               "flop_per_attempt": per_att, "flop_per_accepted": per_acc,
               "peak_source": "derived: 152 SM x 2 FP64 lanes/clk x 2070 MHz, FMA=2 (of derived)"}
    else:
        lookups = 6 * attempted
        gbytes = lookups * (LOOKUP_BYTES[grid_dtype] + (MOD_LOOKUP_BYTES if modulated else 0))
        per_acc = MIXED_FP64_OPS_PER_ACCEPTED + (MIXED_MOD_FP64_OPS_PER_ACCEPTED if modulated else 0)
        ops64 = MIXED_FP64_OPS_PER_ATTEMPT * attempted + per_acc * accepted
        f32 = (MIXED_FP32_FLOP_PER_ATTEMPT + (MIXED_MOD_FP32_FLOP_PER_ATTEMPT if modulated else 0)) * attempted
        t64 = {"achieved": ops64 / prop_s / 1e12, "peak": FP64_OPS_PEAK_T, "unit": "T ops/s",
               "ops_per_attempt": MIXED_FP64_OPS_PER_ATTEMPT, "ops_per_accepted": per_acc,
               "peak_source": "derived: FP64 pipe 152 SM x 2 lanes/clk x 2070 MHz (of derived)"}
    gather = {"achieved": gbytes / prop_s / 1e9, "unit": "GB/s",
              "bytes_per_lookup": gbytes / max(lookups, 1.0), "lookups": lookups,
              "level": "l2" if in_l2 else "hbm"}
    if in_l2:
        gather.update(peak=peaks["l2_gbs"], peak_source="L2-resident copy measured in this run (of measured)")
    else:
        gather.update(peak=peaks["hbm_gbs"], peak_source=peaks["hbm_source"])
    t32 = {"achieved": f32 / prop_s / 1e12, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
           "flop_per_attempt": f32 / max(attempted, 1.0),
           "peak_source": "derived: 152 SM x 128 FP32 lanes/clk x 2070 MHz, FMA=2 (of derived)"}
    terms = {"gather": gather, "fp32": t32, "fp64": t64}
    for t in terms.values():
        t["frac"] = t["achieved"] / t["peak"]
    return terms


def roofline_from_terms(terms, traffic, kernel, note=None):
    """The roofline object of a kernel: the bound is the term closest to its peak (the max
    over the terms, not their sum); every term is kept beside it."""
    name = max(terms, key=lambda k: terms[k]["frac"])
    t = terms[name]
    bound = t["level"] if name == "gather" else "alu"
    out = {"bound": bound, "term": name, "achieved": t["achieved"], "peak": t["peak"], "unit": t["unit"],
           "frac": t["frac"], "traffic": traffic, "kernel": kernel, "peak_source": t["peak_source"],
           "terms": terms}
    if note:
        out["note"] = note
    return out


def roofline_for(form, attempted, accepted, tables, prop_s, calls=1, workload="", modulated=False,
                 grid_dtype="f32", grid_bytes=0, peaks=None, note=None):
    """Roofline of the propagate kernel for one form, from the live CUDA-event time."""
    terms = roofline_terms(form, attempted, accepted, tables, prop_s, modulated, grid_dtype,
                           grid_bytes, peaks)
    kern = ("k_propagate_fp64" if form == "fp64" else "k_propagate_mixed") + \
        " (2 launches per call + 4 bookkeeping kernels)"
    return roofline_from_terms(terms, traffic_for(workload, form, attempted, calls), kern, note)


def deflection_deg(d, sel=None):
    u = np.stack([d["ux"], d["uy"], d["uz"]], 1)
    u0 = np.stack([d["u0x"], d["u0y"], d["u0z"]], 1)
    if sel is not None:
        u, u0 = u[sel], u0[sel]
    return np.degrees(np.arctan2(np.linalg.norm(np.cross(u, u0), axis=1), np.sum(u * u0, 1)))


def mixed_error_statement(w, mixed_state, oracle_state):
    """Precision form vs the FP64 oracle on the oracle sample at full distance: two-sample KS
    on the deflection angle and the log arrival energy of the sampled primaries, overall and
    per primary species (charge)."""
    from scipy import stats

    sel_m = mixed_state["uid"] < 2 ** 32
    sel_o = oracle_state["uid"] < 2 ** 32
    n_s = int(np.sum(sel_o))
    out = {"sample_primaries": n_s, "distance_mpc": w.dmax_m / I.MPC,
           "ks_p_deflection": float(stats.ks_2samp(deflection_deg(mixed_state, sel_m),
                                                   deflection_deg(oracle_state, sel_o)).pvalue),
           "ks_p_log_energy": float(stats.ks_2samp(np.log10(mixed_state["E"][sel_m]),
                                                   np.log10(oracle_state["E"][sel_o])).pvalue)}
    # primaries keep their uid; their species at injection is the charge of the oracle's
    # primary with that uid plus the protons it lost, so split by the injected charge
    zs = sorted(set(int(z) for z in mixed_state.get("Z0", mixed_state["Z"])[sel_m]))
    if "Z0" in mixed_state and len(zs) > 1:
        per = {}
        for z in zs:
            a = sel_m & (mixed_state["Z0"] == z)
            b = sel_o & (oracle_state["Z0"] == z)
            if a.sum() > 20 and b.sum() > 20:
                per[str(z)] = float(stats.ks_2samp(deflection_deg(mixed_state, a),
                                                   deflection_deg(oracle_state, b)).pvalue)
        out["ks_p_deflection_by_primary_charge"] = per
    out["note"] = ("per-particle angles are chaotic beyond ~15 Mpc (1-ulp floor): per-particle error "
                   "by distance is in the by-distance statement")
    return out


def angle_deg(a, b):
    c = np.cross(a, b)
    return np.degrees(np.arctan2(np.linalg.norm(c, axis=1), np.sum(a * b, axis=1)))


def precision_error_by_distance(crp, w, fields, tabs, parts, idx,
                                distances_mpc=(1.0, 2.0, 5.0, 10.0, 20.0)):
    """Arrival-direction error of the precision form against the FP64 form on the GPU (which
    the parity tests hold bit-identical to the FP64 oracle), per primary, at several
    distances, next to the chaos floor (the FP64 form against itself with u0 moved by one ulp
    in x). Each distance is a fresh run of the primaries `idx`."""
    sub = parts.take(np.asarray(idx))
    bumped = sub.take(np.arange(len(sub)))
    bumped.u[:, 0] = np.nextafter(bumped.u[:, 0], 2.0)
    box = I.workload_box(w)
    out = {"sample_primaries": len(sub), "reference": "FP64 form on the GPU (bit-identical to the FP64 oracle)",
           "distances_mpc": [d for d in distances_mpc if d * I.MPC <= w.dmax_m],
           "median_deg": [], "p95_deg": [], "max_deg": [], "chaos_floor_median_deg": [],
           "chaos_floor_p95_deg": [],
           # both forms against a finer FP64 reference (tolerance / 10): how far each is from the
           # trajectory the method converges to, at the workload's tolerance
           "fine_reference": "FP64 form at tolerance / 10", "fp64_vs_fine_p95_deg": [],
           "precision_vs_fine_p95_deg": [], "fp64_vs_fine_median_deg": [], "precision_vs_fine_median_deg": []}

    def final_u(p, form, dmax, tol=None):
        sim = crp.Simulation(fields, tabs, seed=w.rng_seed, capacity=capacity_for(p))
        if box is not None:
            sim.set_boundary(box)
        if w.spectrum is not None:
            sim.sample_sources(crp.Spectrum.of(*w.spectrum), p.x)
        else:
            sim.inject(p)
        sim.propagate(w.tol if tol is None else tol, w.hmin_m, w.hmax_m, dmax, form=form)
        sim.sync(timeout_s=600.0, raise_on_error=False)
        d = sim.state()
        prim = d["uid"] < 2 ** 32
        order = np.argsort(d["uid"][prim])
        return np.stack([d["ux"], d["uy"], d["uz"]], 1)[prim][order]

    for dist in out["distances_mpc"]:
        ref = final_u(sub, crp.FORM_FP64, dist * I.MPC)
        mix = final_u(sub, crp.FORM_MIXED, dist * I.MPC)
        floor_ = final_u(bumped, crp.FORM_FP64, dist * I.MPC) if w.spectrum is None else ref
        e = angle_deg(ref, mix)
        f = angle_deg(ref, floor_)
        fine = final_u(sub, crp.FORM_FP64, dist * I.MPC, tol=w.tol / 10.0)
        ef, em = angle_deg(fine, ref), angle_deg(fine, mix)
        out["fp64_vs_fine_p95_deg"].append(float(np.quantile(ef, 0.95)))
        out["precision_vs_fine_p95_deg"].append(float(np.quantile(em, 0.95)))
        out["fp64_vs_fine_median_deg"].append(float(np.median(ef)))
        out["precision_vs_fine_median_deg"].append(float(np.median(em)))
        out["median_deg"].append(float(np.median(e)))
        out["p95_deg"].append(float(np.quantile(e, 0.95)))
        out["max_deg"].append(float(e.max()))
        out["chaos_floor_median_deg"].append(float(np.median(f)))
        out["chaos_floor_p95_deg"].append(float(np.quantile(f, 0.95)))
    ok = [d for d, p95 in zip(out["distances_mpc"], out["p95_deg"]) if p95 <= 0.1]
    out["p95_within_0p1deg_up_to_mpc"] = max(ok) if ok else None
    if w.spectrum is not None:
        out["note"] = "sources drawn on the device: the chaos floor is not measured for this workload"
    return out


# ---------------------------------------------------------------------------------------
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = workload_for(args)
    n = args.n_particles or w.n_particles
    grids, tables, parts = build_inputs(w, n, 0)
    import oracle as O

    per_step = max(1, args.cpu_sample)
    times, steps_acc = [], []
    for it in range(args.warmup + args.steps):
        lo = (it * per_step) % max(1, len(parts) - per_step)
        if w.spectrum is not None:
            sub = oracle_sources(w, parts, lo, per_step, w.rng_seed)
        else:
            sub = parts.take(np.arange(lo, lo + per_step) if w.n_grids == 1 else
                             np.random.default_rng(it).choice(len(parts), per_step, replace=False))
        st = O.OracleState(capacity_for(sub))
        ot = O.OracleTables(tables) if tables is not None else None
        O.inject(st, sub, w.rng_seed, ot)
        t0 = time.perf_counter()
        rc, stats = O.propagate(st, [g.oracle_field(O, w.spacing_m) for g in grids], ot, w.tol,
                                w.hmin_m, w.hmax_m, w.dmax_m, seed=w.rng_seed,
                                n_threads=os.cpu_count() or 1, box=I.workload_box(w))
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
            steps_acc.append(stats["accepted"])
    value = sum(steps_acc) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "batch_per_step": per_step,
                   "note": "FP64 CPU oracle on a bounded sample of the workload per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count() or 1,
                         "kind": "oracle",
                         "sample": f"{per_step} primaries per step (+ secondaries), full distance"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


_PEAKS = None


def peaks_for(dev) -> dict:
    """Measured HBM peak (file) and L2 copy bandwidth (measured once in this process)."""
    global _PEAKS
    if _PEAKS is None:
        _PEAKS = measured_peaks()
        _PEAKS["l2_gbs"] = measure_l2_gbs(dev)
    return _PEAKS


def grid_read_bytes(sim, crp, fields, grids, form: str, bf16: bool) -> int:
    """Bytes of the grid copy a form reads: the FP64 form its widened copy (32 B per node),
    the precision form the cell-major copy (8 corners per cell) or the node grid."""
    nodes = sum(int(np.prod(f.shape)) for f in fields)
    mod = sum(int(g.mod.size) * 4 for g in grids if g.mod is not None)
    if form == "fp64":
        return nodes * 32 + mod
    if sim.grid_layout() == crp.GRID_CELLS:
        return nodes * (64 if bf16 else 96) + mod
    return nodes * (8 if bf16 else 16) + mod


def with_injected_charge(d: dict, parts) -> dict:
    """Adds Z0, the injected charge of each primary (looked up by uid; -1 for secondaries)."""
    uid = d["uid"]
    prim = uid < 2 ** 32
    pos = np.searchsorted(parts.uid, uid[prim])
    z0 = np.full(len(uid), -1, dtype=np.int32)
    z0[prim] = parts.Z[np.clip(pos, 0, len(parts) - 1)]
    d = dict(d)
    d["Z0"] = z0
    return d


def run_own(args):
    """One workload through the library; returns the JSON line (rank 0 prints it)."""
    import torch

    import paper_1410_5323_gb300 as crp

    ws, rank, local = dist_env()
    dist = None
    if ws > 1 and not getattr(args, "leg", False):
        import torch.distributed as dist

        if not dist.is_initialized():
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = workload_for(args)
    n = args.n_particles or w.n_particles
    grids, tables, parts = build_inputs(w, n, rank)
    n = len(parts)
    cap = capacity_hint(w, parts)
    bf16 = w.bf16

    fields = [g.field(crp, w.spacing_m) for g in grids]
    tabs = crp.Tables(tables) if tables is not None else None
    # device-drawn sources: each rank its own Philox key (uids restart at 0 on every rank)
    seed = w.rng_seed + (1000003 * rank if w.spectrum is not None else 0)
    sim = crp.Simulation(fields, tabs, seed=seed, capacity=cap)
    box = I.workload_box(w)
    if box is not None:
        sim.set_boundary(box)
    slice_steps = args.slice_steps if args.slice_steps >= 0 else (16000 if w.n_grids > 1 else 0)
    grid_bytes = sum(int(np.prod(f.shape)) for f in fields) * (8 if bf16 else 16)
    grid_bytes += sum(int(g.mod.size) * 4 for g in grids if g.mod is not None)
    order = args.order or (3 if w.n_grids > 1 else 2)
    stream = torch.cuda.current_stream(dev)
    peaks = peaks_for(dev)

    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    cols = dict(x=(d(parts.x[:, 0]), d(parts.x[:, 1]), d(parts.x[:, 2])),
                u=(d(parts.u[:, 0]), d(parts.u[:, 1]), d(parts.u[:, 2])),
                E=d(parts.E), A=d(parts.A), Z=d(parts.Z), uid=d(parts.uid), grid_id=d(parts.grid_id))
    form_id = {"fp64": crp.FORM_FP64, "mixed": crp.FORM_MIXED}
    spec = crp.Spectrum.of(*w.spectrum) if w.spectrum is not None else None
    amap = (torch.zeros(12 * w.arrival_nside ** 2, dtype=torch.int64, device=dev)
            if w.arrival_nside else None)

    def add_sources(c):
        if spec is not None:
            sim.sample_sources(spec, c["x"], stream=stream)
        else:
            sim.inject(**c, stream=stream)

    def bin_arrivals():
        if amap is not None:
            amap.zero_()
            sim.arrival_map(w.arrival_nside, w.arrival_emin_ev, out=amap, stream=stream)

    def run_propagate(prm):
        if slice_steps > 0:
            sim.propagate_loop(w.tol, w.hmin_m, w.hmax_m, w.dmax_m, max_steps=slice_steps,
                               stream=stream, **prm)
        else:
            sim.propagate(w.tol, w.hmin_m, w.hmax_m, w.dmax_m, stream=stream, **prm)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2

    def barrier():
        if dist is not None:
            dist.barrier()

    def one_step(form):
        prm = dict(form=form_id[form], block_size=args.block_size, cadence=args.cadence, order=order)
        sim.reset()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        p0 = torch.cuda.Event(enable_timing=True)
        p1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        add_sources(cols)
        p0.record(stream)
        run_propagate(prm)
        p1.record(stream)
        bin_arrivals()
        e1.record(stream)
        rc = sim.sync(0.0, raise_on_error=False)
        c = sim.counts()
        return e0.elapsed_time(e1), p0.elapsed_time(p1), c, rc

    def measure(form, with_clocks):
        for _ in range(args.warmup):
            flush.zero_()
            one_step(form)
        clocks = ClockSampler(local) if with_clocks else None
        barrier()
        torch.cuda.synchronize()
        runs0 = crp.kernel_runs()
        if clocks:
            clocks.start()
        r = dict(step_ms=[], prop_ms=[], accepted=0, attempted=0, rcs=[], secondaries=0, launches=0)
        for _ in range(args.steps):
            flush.zero_()
            ms, pms, c, rc = one_step(form)
            r["step_ms"].append(ms)
            r["prop_ms"].append(pms)
            r["accepted"] += c["accepted"]
            r["attempted"] += c["attempted"]
            r["secondaries"] += c["secondaries"]
            r["launches"] += c["launches"]
            r["rcs"].append(rc)
        torch.cuda.synchronize()
        r["kernel_runs"] = crp.kernel_runs() - runs0
        barrier()
        r["clocks"] = clocks.stop() if clocks else None
        r["total_ms_max"], r["accepted_all"], r["attempted_all"] = aggregate(
            dist, sum(r["step_ms"]), r["accepted"], r["attempted"], dev)
        r["value"] = r["accepted_all"] / (r["total_ms_max"] * 1e-3)
        return r

    main = measure(args.form, True)
    other_form = "mixed" if args.form == "fp64" else "fp64"
    other = None if args.no_other_form else measure(other_form, False)
    # the error statement needs mixed-form results in the simulation state
    last_is_mixed = (other is not None and other_form == "mixed") or (other is None and args.form == "mixed")
    if not last_is_mixed and args.form == "mixed":
        one_step("mixed")
        last_is_mixed = True
    sample_idx = oracle_sample_index(w, n, args.cpu_sample)
    last_state = ({k: sim.read(k, 0, int(sample_idx[-1]) + 1)[sample_idx] for k in crp.COLUMNS}
                  if last_is_mixed else None)
    mixed_layout = sim.grid_layout()

    value = main["value"]
    clk = main["clocks"]
    accepted, attempted, secondaries = main["accepted"], main["attempted"], main["secondaries"]
    accepted_all, attempted_all = main["accepted_all"], main["attempted_all"]
    total_ms_max, rcs = main["total_ms_max"], main["rcs"]
    prop_ms = main["prop_ms"]
    prm = dict(form=form_id[args.form], block_size=args.block_size, cadence=args.cadence, order=order)

    # ---- roofline of the dominant kernel (the propagate call, timed live) ----
    prop_s = sum(prop_ms) * 1e-3
    modulated = bool(w.mod_n)
    gdt = "bf16" if bf16 else "f32"
    note_mixed = ("algorithmic gather volume; L1/L2 serve most of it (measured DRAM bytes per attempt "
                  "in `traffic`); the kernel's limiter is the latency of six dependent lookups per attempt")
    roofline = roofline_for(args.form, attempted, accepted, tables is not None, prop_s,
                            calls=args.steps, workload=w.name, modulated=modulated, grid_dtype=gdt,
                            grid_bytes=grid_read_bytes(sim, crp, fields, grids, args.form, bf16),
                            peaks=peaks, note=note_mixed if args.form == "mixed" else None)

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hcols = dict(x=(pin(parts.x[:, 0]), pin(parts.x[:, 1]), pin(parts.x[:, 2])),
                     u=(pin(parts.u[:, 0]), pin(parts.u[:, 1]), pin(parts.u[:, 2])),
                     E=pin(parts.E), A=pin(parts.A), Z=pin(parts.Z), uid=pin(parts.uid),
                     grid_id=pin(parts.grid_id))
        if spec is not None:         # only positions go up; the arrival map comes back
            hcols = {"x": hcols["x"]}
        h2d = sum(int(t.numel() * t.element_size()) for v in hcols.values()
                  for t in (v if isinstance(v, tuple) else (v,)))
        out = sim.observe_buffers(cap, pinned=True) if amap is None else None
        hmap = torch.empty_like(amap, device="cpu").pin_memory() if amap is not None else None
        # the observer's buffers are set up once, like the pinned inputs: one untimed fill
        # takes the first device write into the new page-locked pages (about 0.1 s for
        # 1.6 GB here) out of the steady-state steps
        if out is not None:
            sim.observe(out=out)
        elif hmap is not None:
            hmap.copy_(amap)
        e2e_times, e2e_steps, d2h = [], 0, 0
        n_e2e = max(1, min(args.steps, args.e2e_steps))
        for _ in range(n_e2e):          # the device path is already warm
            sim.reset()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            add_sources(hcols)
            run_propagate(prm)
            if amap is not None:
                bin_arrivals()
                hmap.copy_(amap, non_blocking=True)
                sim.sync(0.0, raise_on_error=False)
                torch.cuda.synchronize()
                d2h = int(hmap.numel() * hmap.element_size())
            else:
                sim.sync(0.0, raise_on_error=False)
                rec = sim.observe(out=out)
                d2h = sim.observe_bytes(len(rec["uid"]))
            e2e_times.append(time.perf_counter() - t0)
            e2e_steps += sim.counts()["accepted"]
        e2e = {"value": e2e_steps / sum(e2e_times), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": n_e2e}

    cpu, forms, forms_err = None, None, None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu, oracle_state = cpu_baseline(w, grids, tables, parts, args.cpu_sample, "FP64")
        cpu.pop("rc", None)
        if last_state is not None:
            forms_err = mixed_error_statement(w, with_injected_charge(last_state, parts),
                                              with_injected_charge(oracle_state, parts))
    by_distance = None
    if rank == 0 and ws == 1 and last_is_mixed and not args.no_cpu_baseline:
        bd_idx = (oracle_sample_index(w, n, min(args.cpu_sample, 16384)) if w.n_grids > 1
                  else np.arange(min(n, 16384 if not bf16 else 4096)))
        dists = (1.0, 2.0, 5.0, 10.0, 20.0) if not bf16 else (1.0, 2.0, 5.0)
        by_distance = precision_error_by_distance(crp, w, fields, tabs, parts, bd_idx, dists)
    if other is not None:
        forms = {args.form: {"value": value, "unit": UNIT},
                 other_form: {"value": other["value"], "unit": UNIT,
                              "reject_frac": 1.0 - other["accepted_all"] / max(other["attempted_all"], 1.0),
                              "roofline": roofline_for(
                                  other_form, other["attempted"], other["accepted"], tables is not None,
                                  sum(other["prop_ms"]) * 1e-3, calls=args.steps, workload=w.name,
                                  modulated=modulated, grid_dtype=gdt,
                                  grid_bytes=grid_read_bytes(sim, crp, fields, grids, other_form, bf16),
                                  peaks=peaks, note=note_mixed if other_form == "mixed" else None)},
                 "mixed_over_fp64": (other["value"] / value) if other_form == "mixed" else (value / other["value"]),
                 "mixed_error_vs_fp64_oracle": forms_err,
                 "mixed_error_vs_fp64_by_distance": by_distance}

    # the library's kernels that ran in the timed region, counted on the device
    gpu_launches = int(main["kernel_runs"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
        "scaling": "strong" if w.n_grids > 1 else "weak", "vs_baseline": None,
        "dtype": "f64" if args.form == "fp64" else "f32 stages / f64 norm+path / double-float position",
        "data": "synthetic",
        "config": {"workload": w.name, "particles_per_gpu": n,
                   "grid": f"{w.n_grids} x {w.grid_n}^3 " + ("bf16 + fp32 scale" if bf16 else "f32")
                           + (f" x modulation {w.mod_n}^3 f32 ({w.mod_spacing_m / I.KPC:.0f} kpc; vector "
                              f"{w.spacing_m / I.KPC:.0f} kpc)" if w.mod_n else ""),
                   "order": order,
                   "slice_steps": slice_steps,
                   "form": args.form, "dmax_mpc": w.dmax_m / I.MPC, "tol": w.tol,
                   "precision_form_grid_layout": (None if args.form != "mixed" and other is None else
                                                  "cells (8 corners per cell, 256-bit loads)"
                                                  if mixed_layout == crp.GRID_CELLS else "nodes"),
                   "boundary": "reflective box of the modulation volume" if box is not None else "none",
                   "sources": ("Eq. 1 drawn on the device: H, He-4, N-14, Fe-56, x = 1, 0.5, 0.3, 0.1, "
                               "alpha 1.8, R_cut 10^19.8 V, 1e18-1e21 eV, density-weighted positions")
                   if spec is not None else "given columns",
                   "arrival_map": (f"HEALPix RING nside {w.arrival_nside}, E > 10^18.7 eV, every step"
                                   if amap is not None else None),
                   "l2": f"inputs larger than L2 (grids {grid_bytes / 1e6:.0f} MB in device layout, "
                         f"particle state {cap * 140 / 1e9:.2f} GB at 140 B per slot) and a 256 MB flush "
                         f"before every step",
                   "parallelism": (f"dp{ws} (the {w.n_grids} realisations split by grid id: each GPU "
                                   f"holds its own grids and their particles)" if w.n_grids > 1 else
                                   f"dp{ws} (independent particle batches per GPU)")},
        "accepted_steps_per_step": accepted_all / args.steps,
        "attempted_steps_per_step": attempted_all / args.steps,
        "reject_frac": 1.0 - accepted_all / max(attempted_all, 1.0),
        "secondaries_per_step": secondaries / args.steps,
        "arrival_events_per_step": int(amap.sum()) if amap is not None else None,
        "sync_codes": sorted(set(rcs)),
        "roofline": roofline,
        "forms": forms,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": gpu_launches,
        "clocks": clk,
    }
    if other is None and (forms_err is not None or by_distance is not None):
        line["error_vs_fp64_oracle"] = forms_err
        line["error_vs_fp64_by_distance"] = by_distance
    if dist is not None:
        dist.destroy_process_group()
    return line


# Algorithmic FP64 work of the differentiation form per frozen step (FMA = 2): the recorded
# forward is the propagation module (743 per attempt + 83 per accepted step, as the FP64
# form); the backward recomputes the step's stage states (k1..k5: 5 x 81, stage sums 186) and
# reverses it: 6 vector-Jacobian products of f (lookup with weights and their derivatives 129,
# B-bar and u x B 18, kappa-bar 5, u-bar 12, 8 corners x (g . B-bar 5, x-bar 6, 3 scattered
# products 3) = 112 -> 276 each), the stage cotangents (6 x 6 scalings, 15 x 6 x 2 updates
# 180) and the sum 36.
ADJ_FLOP_PER_STEP_BACKWARD = (5 * 81 + 186) + 6 * 276 + 36 + 180 + 36
# Gathered bytes per frozen step: forward 5 lookups per attempt + 1 per step; backward 5 (stage
# states) + 6 (reverse, 8 corners of FP64 values) lookups and 6 x 8 x 3 scattered FP64 adds.
ADJ_SCATTER_BYTES_PER_STEP = 6 * 8 * 3 * 8


def run_adjoint(args):
    """Differentiation workload: record the steps of n particles, then the reverse pass.
    value = frozen steps differentiated per second (n x n_steps / (forward + backward))."""
    import torch

    import oracle as O
    import paper_1410_5323_gb300 as crp
    from paper_1410_5323_gb300.adjoint import Adjoint, direction_loss, perturbed_targets

    ws, rank, local = dist_env()
    dist = None
    if ws > 1 and not getattr(args, "leg", False):
        import torch.distributed as dist

        if not dist.is_initialized():
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    w = workload_for(args)
    n_all = args.n_particles or w.n_particles
    n_steps, K = 2000, 64
    g = I.kolmogorov_grid(w.grid_n, w.spacing_m, w.lmin_cells, w.lmax_cells, w.brms_t,
                          w.grid_seed).astype(np.float32)
    # the job's chains split into blocks over the ranks; dL/dB is summed over them
    lo, hi = shard.block_range(n_all, rank, ws)
    p = I.make_particles(n_all, w.particle_seed, w.species, w.energy).take(np.arange(lo, hi))
    n = len(p)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    peaks = peaks_for(dev)
    field = crp.Field(torch.from_numpy(g).to(dev), w.spacing_m)
    adj = Adjoint(field, n, n_steps, K)
    x0 = torch.from_numpy(p.x).to(dev)
    p0 = torch.from_numpy(p.u * p.E[:, None]).to(dev)
    Z = torch.from_numpy(p.Z).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    clocks = ClockSampler(local)
    fwd_ms, bwd_ms = [], []
    runs0 = 0
    for it in range(args.warmup + args.steps):
        if it == args.warmup:
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize()
            runs0 = crp.kernel_runs()
            clocks.start()
        flush.zero_()
        e0, e1, e1b, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
        e0.record()
        _, uT = adj.forward(x0, p0, Z, w.tol, w.hmin_m, w.hmax_m)
        e1.record()
        t = perturbed_targets(uT)
        u = uT.clone().requires_grad_(True)
        direction_loss(u, t).backward()
        e1b.record()
        gb, pb, xb = adj.backward(u.grad, g.shape)
        shard.allreduce_sum_(gb, dist)
        e2.record()
        torch.cuda.synchronize()
        if it >= args.warmup:
            fwd_ms.append(e0.elapsed_time(e1))
            bwd_ms.append(e1b.elapsed_time(e2))
    runs = crp.kernel_runs() - runs0
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    steps = n * n_steps
    t_max, steps_all, _ = aggregate(dist, (sum(fwd_ms) + sum(bwd_ms)), float(steps * args.steps), 0.0, dev)
    t_s = (sum(fwd_ms) + sum(bwd_ms)) * 1e-3
    value = steps_all / (t_max * 1e-3)
    h = adj.steps().cpu().numpy()
    # attempts of the recorded forward are not counted by the kernel: a step is one attempt
    # when no rejection happened, which the recorded sizes show (h equals the proposal).
    att_per_step = 1.0
    fl = (FLOP_PER_ATTEMPT * att_per_step + FLOP_PER_ACCEPTED + ADJ_FLOP_PER_STEP_BACKWARD) * steps * args.steps
    lookups = (5 * att_per_step + 1 + 5 + 6) * steps * args.steps
    gbytes = lookups * LOOKUP_BYTES["f64"] + ADJ_SCATTER_BYTES_PER_STEP * steps * args.steps
    grid_copy = int(np.prod(g.shape[:3])) * 32
    in_l2 = grid_copy <= L2_BYTES
    terms = {
        "gather": {"achieved": gbytes / t_s / 1e9, "unit": "GB/s", "level": "l2" if in_l2 else "hbm",
                   "peak": peaks["l2_gbs"] if in_l2 else peaks["hbm_gbs"],
                   "peak_source": ("L2-resident copy measured in this run (of measured)" if in_l2
                                   else peaks["hbm_source"]),
                   "bytes_per_frozen_step": gbytes / (steps * args.steps)},
        "fp64": {"achieved": fl / t_s / 1e12, "unit": "TFLOP/s", "peak": FP64_PEAK_TFLOPS,
                 "flop_per_frozen_step": fl / (steps * args.steps),
                 "peak_source": "derived: 152 SM x 2 FP64 lanes/clk x 2070 MHz, FMA=2 (of derived)"},
    }
    for tt in terms.values():
        tt["frac"] = tt["achieved"] / tt["peak"]
    roof = roofline_from_terms(terms, None,
                               "k_adj_record_team + k_adj_records + k_adj_reverse_team (+ init, p0-bar)",
                               note=f"{n} independent chains: three lanes per chain (one per axis) in the "
                                    "serial record and reverse sweeps, one thread per (chain, segment) "
                                    "in the stage records")

    # ---- end to end: inputs from pinned host memory, gradients back ----
    hx0 = torch.from_numpy(p.x).pin_memory()
    hp0 = torch.from_numpy(p.u * p.E[:, None]).pin_memory()
    hZ = torch.from_numpy(p.Z).pin_memory()
    hgb = torch.empty(tuple(g.shape[:3]) + (3,), dtype=torch.float64).pin_memory()
    hpb = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    e2e_t = []
    n_e2e = max(1, min(args.steps, args.e2e_steps))
    for _ in range(n_e2e):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dx0, dp0, dZ = hx0.to(dev, non_blocking=True), hp0.to(dev, non_blocking=True), hZ.to(dev, non_blocking=True)
        _, uT = adj.forward(dx0, dp0, dZ, w.tol, w.hmin_m, w.hmax_m)
        t = perturbed_targets(uT)
        u = uT.clone().requires_grad_(True)
        direction_loss(u, t).backward()
        gb, pb, _ = adj.backward(u.grad, g.shape)
        hgb.copy_(gb, non_blocking=True)
        hpb.copy_(pb, non_blocking=True)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    e2e = {"value": steps * n_e2e / sum(e2e_t), "unit": "steps/s",
           "h2d_bytes_per_step": int(hx0.numel() * 8 + hp0.numel() * 8 + hZ.numel() * 4),
           "d2h_bytes_per_step": int(hgb.numel() * 8 + hpb.numel() * 8), "steps": n_e2e}

    # ---- error statement: reverse pass vs the oracle's, central differences ----
    err, cpu = None, None
    if not args.no_cpu_baseline and ws == 1:
        _, uT = adj.forward(x0, p0, Z, w.tol, w.hmin_m, w.hmax_m)
        t = perturbed_targets(uT)
        un = torch.linalg.norm(uT, dim=1, keepdim=True)
        uh = uT / un
        gu = 2 * (uh - t)
        lam = ((gu - uh * (uh * gu).sum(1, keepdim=True)) / un).cpu().numpy()
        gb, pb, xb = adj.backward(torch.from_numpy(lam), g.shape)
        pb, xb = pb.cpu().numpy(), xb.cpu().numpy()
        pick = np.sort(np.random.default_rng(0).choice(n, 8, replace=False))
        sub = Adjoint(field, len(pick), n_steps, K)
        sub.forward(x0[pick], p0[pick], Z[pick], w.tol, w.hmin_m, w.hmax_m)
        gbs = sub.backward(torch.from_numpy(lam[pick]), g.shape)[0].cpu().numpy()
        of = O.OracleField(g, w.spacing_m)
        go = np.zeros(g.shape)
        p0n = p.u * p.E[:, None]
        E = np.sqrt((p0n[:, 0] * p0n[:, 0] + p0n[:, 1] * p0n[:, 1]) + p0n[:, 2] * p0n[:, 2])
        u0 = p0n / E[:, None]
        kap = (p.Z.astype(np.float64) * 299792458.0) / E
        same_steps = same_x0 = same_p0 = 0
        t0 = time.perf_counter()
        for i in pick:
            y0 = np.concatenate([p.x[i], u0[i]])
            ho, _ = O.record_steps(of, kap[i], y0, w.tol, w.hmin_m, w.hmax_m, n_steps)
            yb, kb = O.adjoint(of, kap[i], y0, ho, np.concatenate([np.zeros(3), lam[i]]), go)
            same_steps += int(np.array_equal(h[:, i], ho))
            same_x0 += int(np.array_equal(xb[i], yb[:3]))
            dot = (u0[i, 0] * yb[3] + u0[i, 1] * yb[4]) + u0[i, 2] * yb[5]
            same_p0 += int(np.array_equal(pb[i], (yb[3:] - dot * u0[i]) / E[i] + (-(kb * kap[i]) / E[i]) * u0[i]))
        dt = time.perf_counter() - t0
        nz = np.abs(go) > 1e-12 * np.abs(go).max()
        rel = float(np.max(np.abs(gbs[nz] - go[nz]) / np.abs(go[nz])))
        err = {"oracle_reverse_pass": {"sampled_particles": len(pick), "frozen_steps": n_steps,
                                       "steps_bit_identical": same_steps, "x0_grad_bit_identical": same_x0,
                                       "p0_grad_bit_identical": same_p0,
                                       "grid_grad_max_rel_diff": rel}}
        err["central_differences"] = adjoint_fd_check(crp, Adjoint, direction_loss, perturbed_targets,
                                                      w, g, field, x0, p0, Z)
        cpu = {"value": len(pick) * n_steps / dt, "unit": "steps/s", "cores": 1, "kind": "oracle",
               "sample": f"{len(pick)} of the {n} chains: recorded forward + reverse pass over "
                         f"{n_steps} frozen steps in {dt:.2f} s (FP64 oracle, one thread)"}
    if dist is not None and not getattr(args, "leg", False):
        dist.destroy_process_group()
    return {
        "metric": "frozen particle-steps differentiated/s (recorded forward + checkpointed reverse pass)",
        "value": value, "unit": "steps/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "particles": n_all, "particles_per_gpu": n, "frozen_steps": n_steps,
                   "checkpoint_every": K, "grid": f"{w.grid_n}^3 f32 (read as its FP64 copy)",
                   "l2": "256 MB flush before every step",
                   "parallelism": f"dp{ws} (chains split in blocks; dL/dB summed by one all-reduce per step)"},
        "forward_ms": sum(fwd_ms) / args.steps, "backward_ms": sum(bwd_ms) / args.steps,
        "roofline": roof, "e2e": e2e, "error_vs_fp64_oracle": err, "cpu_baseline": cpu,
        "gpu_launches": int(runs),          # the library's kernels in the timed region, counted on the device
        "clocks": clk,
    }


def adjoint_fd_check(crp, Adjoint, direction_loss, perturbed_targets, w, g, field, x0, p0, Z,
                     n_steps=200, n_entries=8):
    """Central differences of the loss over the first n_steps frozen steps (the horizon in
    which the chaotic map stays linear at representable eps) on n_entries grid values with a
    large gradient; a difference counts only when its +eps and -eps replays visit the same
    cells as the unperturbed one; two such a decade apart are Richardson-extrapolated."""
    import torch

    adj = Adjoint(field, x0.shape[0], n_steps, 64)
    _, uT = adj.forward(x0, p0, Z, w.tol, w.hmin_m, w.hmax_m)
    t = perturbed_targets(uT)
    u = uT.clone().requires_grad_(True)
    direction_loss(u, t).backward()
    gb, _, _ = adj.backward(u.grad, g.shape)
    gbf = gb.view(-1)
    big = torch.nonzero(gbf.abs() > 1e-3 * gbf.abs().max()).view(-1)
    pick = big[torch.randperm(big.numel(), generator=torch.Generator().manual_seed(0))[:n_entries].to(big.device)]
    g64 = torch.from_numpy(g).to(gb.device).double()
    _, _, h0 = adj.replay(cells=True)

    def central(idx, eps):
        out = []
        for sgn in (1.0, -1.0):
            gp = g64.clone().view(-1)
            gp[idx] += sgn * eps
            _, up, hp = adj.replay(crp.Field(gp.view(g64.shape), w.spacing_m), cells=True)
            if not torch.equal(hp, h0):
                return None
            out.append(direction_loss(up, t))
        return float((out[0] - out[1]) / (2 * eps))

    errs = []
    for idx in pick.tolist():
        ds = [(e, central(idx, e)) for e in (1e-18, 1e-19, 1e-20)]
        fd = None
        for (_, d1), (_, d2) in zip(ds, ds[1:]):
            if d1 is not None and d2 is not None:
                fd = (100.0 * d2 - d1) / 99.0
                break
        if fd is None:
            valid = [d for _, d in ds if d is not None]
            fd = valid[0] if valid else None
        if fd is not None:
            errs.append(abs(fd - float(gbf[idx])) / abs(float(gbf[idx])))
    return {"frozen_steps": n_steps, "grid_entries": len(pick), "checkable": len(errs),
            "max_rel_err": max(errs) if errs else None, "bar": 1e-4}


def run_lens(args):
    """Lens workload (Sec. 3.3): a synthetic nside-64 lens of 24 rigidity bins (24 entries per
    column, 9.4 MB per matrix) applied to rigidity-binned arrival maps. value = stored entries applied per second
    (entries x maps / device time), one fused launch over all bins per step; roofline against
    HBM with the algorithmic bytes of a launch."""
    import torch

    import paper_1410_5323_gb300 as crp

    ws, rank, _ = dist_env()
    nside, n_mat, k = 64, 24, 24
    n_pix = 12 * nside * nside
    n_maps = args.n_maps
    rp, col, val = I.synthetic_lens(nside, I.lens_edges(n_mat), seed=1, k=k)
    nnz = int(col.size)
    lens = crp.Lens(n_pix, rp, col, val)
    if args.lens_group:
        lens.set_group(args.lens_group)
    dev = torch.device("cuda")
    xh = np.random.default_rng(1 + rank).poisson(3.0, (n_mat, n_pix, n_maps)).astype(np.float64)
    x = torch.from_numpy(xh if n_maps > 1 else xh[:, :, 0]).to(dev).contiguous()
    y = torch.empty((n_pix, n_maps) if n_maps > 1 else (n_pix,), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        flush.zero_()
        lens.apply(x, out=y, stream=stream)
    clocks = ClockSampler(0 if ws == 1 else int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.synchronize()
    runs0 = crp.kernel_runs()
    clocks.start()
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lens.apply(x, out=y, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    runs = crp.kernel_runs() - runs0
    clk = clocks.stop()
    t = sum(ms) * 1e-3
    value = nnz * n_maps * args.steps / t
    algo = nnz * 8 + n_mat * (n_pix + 1) * 8 + n_mat * n_pix * n_maps * 8 + n_pix * n_maps * 8
    ach = algo * args.steps / t / 1e9
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    # the launch is bound by the slower of streaming the lens (HBM) and one FP64 FMA per entry
    # and map (GB300's FP64 pipe: 2 lanes/clk/SM); the bound reported is the one that binds
    t_hbm = algo / (peak * 1e9)
    t_fp64 = nnz * n_maps / (FP64_OPS_PEAK_T * 1e12)
    hbm = {"achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak, "algorithmic_bytes": algo,
           "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    kern = "k_lens_apply_vec (one map) / k_lens_apply_maps (several), one launch per step"
    if t_fp64 >= t_hbm:
        fl = 2.0 * nnz * n_maps * args.steps / t / 1e12
        roof = {"bound": "alu", "achieved": fl, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": fl / FP64_PEAK_TFLOPS, "traffic": LENS_DRAM_BYTES.get(n_maps), "kernel": kern,
                "flop_per_entry_and_map": 2,
                "peak_source": "derived: 152 SM x 2 FP64 lanes/clk x 2070 MHz, FMA=2 (of derived)", "hbm": hbm}
    else:
        roof = dict(bound="hbm", traffic=LENS_DRAM_BYTES.get(n_maps), kernel=kern, **hbm)
    # end to end through the binding: maps up from pinned host memory, observed maps back
    xp = torch.from_numpy(xh if n_maps > 1 else np.ascontiguousarray(xh[:, :, 0])).pin_memory()
    yp = torch.empty(tuple(y.shape), dtype=torch.float64).pin_memory()
    xd = torch.empty_like(x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        xd.copy_(xp, non_blocking=True)
        lens.apply(xd, out=y, stream=stream)
        yp.copy_(y, non_blocking=True)
        torch.cuda.synchronize()
    te = time.perf_counter() - t0
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle as O

        t1 = time.perf_counter()
        O.lens_apply(n_pix, rp, col, val, xh[:, :, :1])
        dt = time.perf_counter() - t1
        cpu = {"value": nnz / dt, "unit": "entries/s", "cores": 1, "kind": "oracle",
               "sample": f"the whole lens ({nnz} entries), one map, in {dt:.2f} s (FP64 oracle, one thread)"}
    line = {
        "metric": "lens entries applied/s (stored matrix entries x maps / device time, Sec. 3.3 lens)",
        "value": value, "unit": "entries/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sum(ms) / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 values, f64 products and sums", "data": "synthetic",
        "config": {"workload": "lens_nside64_24bins", "n_pix": n_pix, "rigidity_bins": n_mat,
                   "entries": nnz, "entries_per_column": k, "maps": n_maps,
                   "lens_bytes": int(nnz * 8 + rp.nbytes),
                   "l2": "lens (227 MB) larger than L2 and a 256 MB flush before every step",
                   "parallelism": f"dp{ws} (independent lenses per GPU)"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": nnz * n_maps * args.steps / te, "unit": "entries/s",
                "h2d_bytes_per_step": int(xp.numel() * 8), "d2h_bytes_per_step": int(yp.numel() * 8)},
        "gpu_launches": int(runs),
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# Extra legs of the default run, one per form the method adds: (key, workload, oracle sample).
FORM_LEGS = (("precision_1024cube_bf16", "mixed_1024cube_10M_pFe", 10000),
             ("batched_64x128cube", "batched_64x128cube_12.8M_protons", 6400),
             ("adjoint_128cube", "adjoint_128cube_4k_protons", 0))


def run_leg(args, workload: str, sample: int) -> dict:
    """One extra workload with fewer steps; returns its figures for the headline's `forms`."""
    import copy
    import gc

    import torch

    gc.collect()                       # the previous leg's grids and state are freed
    torch.cuda.empty_cache()
    a = copy.copy(args)
    a.workload, a.leg = workload, True
    a.steps, a.warmup = args.forms_steps, args.forms_warmup
    a.n_particles, a.grid_n, a.slice_steps, a.order = 0, 0, -1, 0
    a.cpu_sample = sample or args.cpu_sample
    if workload.startswith("adjoint"):
        r = run_adjoint(a)
    else:
        a.form, a.no_other_form = "mixed", True
        r = run_own(a)
    gc.collect()
    torch.cuda.empty_cache()
    keep = ("metric", "value", "unit", "steps", "warmup", "ms_per_step", "dtype", "config", "reject_frac",
            "accepted_steps_per_step", "forward_ms", "backward_ms", "roofline", "e2e",
            "error_vs_fp64_oracle", "error_vs_fp64_by_distance", "cpu_baseline", "gpu_launches", "clocks")
    return {k: r[k] for k in keep if k in r}


def main():
    args = parse()
    if args.workload.startswith("lens"):
        return run_lens(args)
    if args.workload.startswith("adjoint"):
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm covers the propagation "
                                                                  "workloads; the adjoint's oracle timing is "
                                                                  "its cpu_baseline"}))
            return 0
        line = run_adjoint(args)
        if dist_env()[1] == 0:
            print(json.dumps(line), flush=True)
        return 0
    w = workload_for(args)
    default_run = args.workload == "fp64_256cube_1M_nuclei" and not args.n_particles and not args.grid_n
    if args.form is None:
        both = w.name.startswith("fp64") or w.mod_n > 0
        args.form = "fp64" if both else "mixed"
        if not both:
            args.no_other_form = True
    if args.impl == "reference":
        return run_reference(args)
    line = run_own(args)
    ws, rank, _ = dist_env()
    if default_run and ws == 1 and not args.no_forms:
        if line.get("forms") is None:
            line["forms"] = {}
        for key, wl, sample in FORM_LEGS:
            line["forms"][key] = run_leg(args, wl, sample)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
