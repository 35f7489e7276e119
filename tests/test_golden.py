"""The synthetic workloads and constants against the numbers the paper prints (fixtures in
tests/golden/, each citing its section): lens sizes (Sec. 3.3) and the Sec. 4 scenario
(modulation and vector grid geometry, coherence length, Eq. 1 parameters, arrival threshold)."""
import math
import os

import numpy as np

from paper_1410_5323_gb300 import inputs as I

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _read(name):
    out = {}
    for line in open(os.path.join(HERE, name)):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = (t.strip() for t in line.split("=", 1))
            out[k] = v
    return out


def test_lens_sizes_sec3_3():
    g = _read("sec3_3_lens_sizes.txt")
    nside = 64
    n_pix = 12 * nside * nside
    assert abs(n_pix - float(g["pixels_approx"])) / float(g["pixels_approx"]) < 0.02
    assert math.degrees(math.sqrt(4 * math.pi / n_pix)) < float(g["angular_resolution_deg_below"])
    assert round(n_pix ** 2 * 4 / 2 ** 30) == int(g["dense_single_precision_gib"])
    rp, col, val = I.synthetic_lens(8, I.lens_edges(2), seed=1)         # default entries per column
    per_entry = col.itemsize + val.itemsize
    k = col.size // (2 * 12 * 8 * 8)
    assert n_pix * k * per_entry / 1e6 < float(g["sparse_matrix_mb_below"])


def test_sec4_scenario_parameters():
    g = _read("sec4_scenario.txt")
    w = I.workload("sec4_eq1_440cube_x_256cube_1M_nuclei")
    assert abs(w.mod_n * w.mod_spacing_m / I.MPC - float(g["modulation_edge_mpc"])) < 1e-9
    assert abs(w.mod_spacing_m / I.KPC - float(g["modulation_resolution_kpc"])) < 1e-9
    assert abs(w.spacing_m / I.KPC - float(g["vector_resolution_kpc"])) < 1e-9
    # coherence length of a Kolmogorov field on [l_min, l_max] (spectral index 5/3 of the energy)
    a = 5.0 / 3.0
    lmin, lmax = w.lmin_cells * w.spacing_m, w.lmax_cells * w.spacing_m
    r = lmin / lmax
    lc = lmax / 2 * (a - 1) / a * (1 - r ** a) / (1 - r ** (a - 1))
    assert abs(lc / I.KPC - float(g["vector_coherence_kpc"])) / float(g["vector_coherence_kpc"]) < 0.02
    species, alpha, rcut, _, _ = w.spectrum
    assert alpha == float(g["eq1_spectral_index"])
    assert abs(math.log10(rcut) - float(g["eq1_log10_cutoff_rigidity_v"])) < 1e-12
    names = {(1, 1): "H-1", (4, 2): "He-4", (14, 7): "N-14", (56, 26): "Fe-56"}
    assert [names[(a_, z)] for a_, z, _ in species] == g["eq1_species"].split()
    assert [x for _, _, x in species] == [float(v) for v in g["eq1_abundances"].split()]
    assert abs(math.log10(w.arrival_emin_ev) - float(g["arrival_log10_energy_threshold_ev"])) < 1e-12
