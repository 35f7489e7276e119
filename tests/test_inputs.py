"""Pins of the seeded synthetic inputs: the Kolmogorov field recipe (paper Sec. 4),
isotropic emission and power-law spectra."""
import math

import numpy as np
from scipy import stats

from paper_1410_5323_gb300 import inputs as I


def _spectrum_of(B):
    n = B.shape[0]
    F = np.stack([np.fft.fftn(B[..., c]) for c in range(3)], -1)
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    kx, ky, kz = np.meshgrid(k1, k1, k1, indexing="ij")
    return F, kx, ky, kz


def test_kolmogorov_per_mode_power_slope_and_band():
    n, lmin, lmax = 32, 2.0, 16.0
    B = I.kolmogorov_grid(n, 1.0, lmin, lmax, 1.0, 7)
    F, kx, ky, kz = _spectrum_of(B)
    kk = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    P = np.sum(np.abs(F) ** 2, -1)
    nyq = (kx == -n // 2) | (ky == -n // 2) | (kz == -n // 2)
    band = (kk >= n / lmax) & (kk <= n / lmin) & ~nyq
    # outside the band (and on Nyquist planes) there is no power
    assert np.max(P[~band]) < 1e-24 * np.max(P)
    # inside, every mode carries |k|^(-11/3) times one common factor
    ratio = P[band] * kk[band] ** (11.0 / 3.0)
    assert np.max(np.abs(ratio / ratio.mean() - 1)) < 1e-9
    slope = np.polyfit(np.log(kk[band]), np.log(P[band]), 1)[0]
    assert abs(slope + 11.0 / 3.0) < 1e-6


def test_kolmogorov_divergence_free_and_rms():
    n = 32
    B = I.kolmogorov_grid(n, 0.5, 2.0, 16.0, 3e-13, 9)
    F, kx, ky, kz = _spectrum_of(B)
    div = kx * F[..., 0] + ky * F[..., 1] + kz * F[..., 2]
    scale = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2) * np.sqrt(np.sum(np.abs(F) ** 2, -1))
    assert np.max(np.abs(div)) < 1e-12 * np.max(scale)
    assert math.sqrt(np.mean(np.sum(B * B, -1))) == __import__("pytest").approx(3e-13, rel=1e-12)
    # the field is real and has zero mean
    assert np.allclose(B.mean(axis=(0, 1, 2)), 0, atol=1e-12 * 3e-13)


def test_kolmogorov_seeded_reproducible():
    a = I.kolmogorov_grid(16, 1.0, 2, 8, 1.0, 3)
    b = I.kolmogorov_grid(16, 1.0, 2, 8, 1.0, 3)
    c = I.kolmogorov_grid(16, 1.0, 2, 8, 1.0, 4)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_isotropic_directions():
    p = I.make_particles(20000, 5)
    assert np.allclose(np.linalg.norm(p.u, axis=1), 1.0, atol=1e-15)
    # each Cartesian component of an isotropic unit vector is uniform on [-1, 1]
    for c in range(3):
        assert stats.kstest(p.u[:, c], "uniform", args=(-1, 2)).pvalue > 1e-3
    assert np.all(p.x == 0)


def test_power_law_and_composition():
    p = I.make_particles(50000, 6, species=(("H", .4), ("He", .3), ("N", .2), ("Fe", .1)),
                         energy=("power", 1e18, 10 ** 20.5, 2.0))
    lo, hi = 1e18, 10 ** 20.5
    assert p.E.min() >= lo and p.E.max() <= hi
    # E^-2 on [lo, hi]: CDF(E) = (1/lo - 1/E)/(1/lo - 1/hi)
    cdf = lambda e: (1 / lo - 1 / e) / (1 / lo - 1 / hi)
    assert stats.kstest(p.E, cdf).pvalue > 1e-3
    fr = np.array([np.mean(p.A == a) for a in (1, 4, 14, 56)])
    assert np.allclose(fr, [.4, .3, .2, .1], atol=0.01)
    assert set(zip(p.A.tolist(), p.Z.tolist())) == {(1, 1), (4, 2), (14, 7), (56, 26)}
    assert np.array_equal(p.uid, np.arange(50000))


def test_log_uniform_energies():
    p = I.make_particles(20000, 8, energy=("loguniform", 1e17, 10 ** 20.5))
    x = np.log10(p.E)
    assert stats.kstest(x, "uniform", args=(17, 3.5)).pvalue > 1e-3


def test_synthetic_table_layout():
    t = I.synthetic_tables()
    assert t.log10_loss.shape == (27 * 31, 201)
    x = I.table_nodes()
    assert x[0] == 6.0 and abs(x[-1] - 14.0) < 1e-14 and abs(x[90] - 9.6) < 1e-14 and abs(x[75] - 9.0) < 1e-14
    assert t.has_loss[t.species_index(1, 0)] == 0 and t.has_pd[t.species_index(1, 1)] == 0
    assert t.has_loss[t.species_index(56, 26)] == 1 and t.has_pd[t.species_index(56, 26)] == 1


def test_torch_kolmogorov_recipe_on_cpu():
    """The device generator used for 1024^3 grids: same band, slope, divergence and rms."""
    torch = __import__("pytest").importorskip("torch")
    n, lmin, lmax = 32, 2.0, 16.0
    B = I.kolmogorov_grid_torch(n, lmin, lmax, 2e-13, 5, device="cpu").double().numpy()
    assert math.sqrt(np.mean(np.sum(B * B, -1))) == __import__("pytest").approx(2e-13, rel=1e-5)
    F, kx, ky, kz = _spectrum_of(B)
    kk = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    P = np.sum(np.abs(F) ** 2, -1)
    nyq = (kx == -n // 2) | (ky == -n // 2) | (kz == -n // 2)
    band = (kk >= n / lmax) & (kk <= n / lmin) & ~nyq
    assert np.max(P[~band]) < 1e-9 * np.max(P)
    ratio = P[band] * kk[band] ** (11.0 / 3.0)
    assert np.max(np.abs(ratio / ratio.mean() - 1)) < 1e-3        # FP32 spectrum
    div = kx * F[..., 0] + ky * F[..., 1] + kz * F[..., 2]
    assert np.max(np.abs(div)) < 1e-5 * np.max(np.sqrt(kk ** 2 * P))


def test_bf16_quantization_scale_is_fp32_and_values_close():
    torch = __import__("pytest").importorskip("torch")
    B = torch.from_numpy(I.kolmogorov_grid(16, 1.0, 2, 8, 3e-13, 2).astype(np.float32))
    q, scale = I.quantize_bf16(B)
    assert q.dtype == torch.bfloat16 and scale == float(np.float32(scale))
    err = (q.float() * scale - B).abs().max() / B.abs().max()
    assert err < 2 ** -8
