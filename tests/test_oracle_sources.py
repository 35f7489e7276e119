"""Pins of the oracle's source spectrum (Sec. 4, Eq. 1), its atan2 and its HEALPix RING
pixelization used for the arrival maps of Sec. 4 (Fig. 4). References: numpy's arctan2, the
HEALPix pixel-centre formulas of Gorski et al. (2005) and its base-pixel layout, equal pixel
areas, closed-form and numerically integrated spectra (scipy), isotropy."""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import oracle as O

EQ1 = [(1, 1, 1.0), (4, 2, 0.5), (14, 7, 0.3), (56, 26, 0.1)]     # (A, Z, x_i), Sec. 4
RCUT = 10 ** 19.8


# ---- atan2 --------------------------------------------------------------------------------
def test_atan2_within_three_ulp_of_numpy(oracle_lib):
    """Error bound of the stated algorithm: 3 ulp of the result (measured maximum over 24k
    points including tiny and huge arguments); a wrong coefficient, sign or octant fails."""
    rng = np.random.default_rng(31)
    pts = list(rng.standard_normal((3000, 2))) + list(10 ** rng.uniform(-300, 300, (500, 2)))
    pts += [(1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (1, -1), (-1, -1), (1e-300, 1),
            (1, 1e-300), (3e200, -2e200), (0.41421356237309503, 1), (1, 0.41421356237309503)]
    for y, x in pts:
        a, b = O.atan2(float(y), float(x)), float(np.arctan2(y, x))
        assert abs(a - b) <= 3 * np.spacing(abs(b)), (y, x, a, b)


# ---- HEALPix -------------------------------------------------------------------------------
def _unit(z, phi):
    s = np.sqrt(1.0 - z * z)
    return np.array([s * np.cos(phi), s * np.sin(phi), z])


def _centres(nside):
    """Pixel centres in RING order from the published formulas (not from the pixelizer):
    north cap ring i < nside: z = 1 - i^2/(3 nside^2), phi = pi/(2i) (j + 1/2), j < 4i;
    belt ring nside <= i <= 3 nside: z = 4/3 - 2i/(3 nside), phi = pi/(2 nside) (j + s/2),
    s = (i - nside + 1) mod 2; south cap mirrors the north one."""
    out = []
    for i in range(1, nside):
        z = 1.0 - i * i / (3.0 * nside * nside)
        out += [_unit(z, math.pi / (2 * i) * (j + 0.5)) for j in range(4 * i)]
    for i in range(nside, 3 * nside + 1):
        z = 4.0 / 3.0 - 2.0 * i / (3.0 * nside)
        s = (i - nside + 1) % 2
        out += [_unit(z, math.pi / (2 * nside) * (j + s / 2.0)) for j in range(4 * nside)]
    for i in range(nside - 1, 0, -1):
        z = -(1.0 - i * i / (3.0 * nside * nside))
        out += [_unit(z, math.pi / (2 * i) * (j + 0.5)) for j in range(4 * i)]
    return np.array(out)


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 16])
def test_pixel_centres_map_to_their_own_index(oracle_lib, nside):
    c = _centres(nside)
    assert len(c) == 12 * nside * nside
    assert np.array_equal(O.healpix_ring(nside, c), np.arange(len(c)))


def test_base_pixels(oracle_lib):
    """The 12 base pixels: 0-3 around the north pole centred at phi = pi/4 + k pi/2 (z = 2/3),
    4-7 on the equator at phi = k pi/2, 8-11 like 0-3 in the south."""
    q = math.pi / 4
    dirs = [_unit(2 / 3, q + k * 2 * q) for k in range(4)] + [_unit(0.0, k * 2 * q) for k in range(4)] + \
           [_unit(-2 / 3, q + k * 2 * q) for k in range(4)]
    assert np.array_equal(O.healpix_ring(1, np.array(dirs)), np.arange(12))
    assert O.healpix_ring(1, [[0, 0, 1]])[0] == 0 and O.healpix_ring(1, [[0, 0, -1]])[0] == 8


def test_equal_areas(oracle_lib):
    rng = np.random.default_rng(32)
    n, nside = 200_000, 4
    u = rng.standard_normal((n, 3))
    counts = np.bincount(O.healpix_ring(nside, u), minlength=12 * nside ** 2)
    assert len(counts) == 192
    assert stats.chisquare(counts).pvalue > 1e-3


def test_scale_invariance_and_invalid_directions(oracle_lib):
    rng = np.random.default_rng(33)
    u = rng.standard_normal((2000, 3))
    assert np.array_equal(O.healpix_ring(8, u), O.healpix_ring(8, 8.0 * u))
    assert O.healpix_ring(8, [[0.0, 0.0, 0.0]])[0] == -1


# ---- Eq. 1 sampler -------------------------------------------------------------------------
def _cdf(alpha, zr, lo, hi):
    """CDF of E^-alpha exp(-E/zr) on [lo, hi] by quadrature in ln E (independent of the sampler)."""
    f = lambda le: math.exp((1 - alpha) * le - math.exp(le) / zr)
    tot = integrate.quad(f, math.log(lo), math.log(hi), limit=200)[0]
    return lambda E: np.array([integrate.quad(f, math.log(lo), math.log(e), limit=200)[0] / tot for e in np.atleast_1d(E)])


def test_pure_power_law_without_cutoff(oracle_lib):
    sp = O.spectrum([(1, 1, 1.0)], 1.8, 1e60, 1e18, 1e21)
    A, Z, E, u, failed = O.source_sample(sp, 7, 0, 40000)
    assert failed == 0 and np.all(A == 1) and np.all(Z == 1)
    g = 1 - 1.8
    cdf = lambda e: (e ** g - 1e18 ** g) / (1e21 ** g - 1e18 ** g)
    assert stats.kstest(E, cdf).pvalue > 0.01
    assert E.min() >= 1e18 and E.max() <= 1e21


def test_log_uniform_when_alpha_is_one(oracle_lib):
    sp = O.spectrum([(1, 1, 1.0)], 1.0, 1e60, 1e18, 1e20)
    _, _, E, _, _ = O.source_sample(sp, 8, 0, 20000)
    assert stats.kstest(np.log(E), "uniform", args=(math.log(1e18), math.log(100.0))).pvalue > 0.01


@pytest.mark.parametrize("A,Z,rcut,emin", [(1, 1, RCUT, 1e18), (4, 2, RCUT, 1e18), (14, 7, 1e19, 1e19),
                                            (56, 26, RCUT, 1e18)])
def test_single_species_cutoff_spectrum(oracle_lib, A, Z, rcut, emin):
    """The cutoff energy is Z R_cut (a rigidity cutoff): with E_min near it, a nucleus with
    A != Z separates it from a cutoff at A R_cut."""
    sp = O.spectrum([(A, Z, 1.0)], 1.8, rcut, emin, 1e21)
    _, _, E, _, failed = O.source_sample(sp, 9, 0, 4000)
    assert failed == 0
    cdf = _cdf(1.8, Z * rcut, emin, 1e21)
    assert stats.kstest(E, cdf).pvalue > 0.01


def test_eq1_species_fractions_and_energies(oracle_lib):
    sp = O.spectrum(EQ1, 1.8, RCUT, 1e18, 1e21)
    n = 60000
    A, Z, E, _, failed = O.source_sample(sp, 10, 0, n)
    assert failed == 0
    f = lambda le, zr: math.exp(-0.8 * le - math.exp(le) / zr)
    w = np.array([x * a ** 0.8 * integrate.quad(f, math.log(1e18), math.log(1e21), args=(z * RCUT,),
                                                limit=200)[0] for a, z, x in EQ1])
    p = w / w.sum()
    counts = np.array([np.sum(A == a) for a, _, _ in EQ1])
    assert counts.sum() == n
    sig = np.sqrt(n * p * (1 - p))
    assert np.all(np.abs(counts - n * p) < 4.5 * sig), (counts, n * p)
    for a, z, _ in EQ1:
        sel = E[A == a][:1500]
        assert stats.kstest(sel, _cdf(1.8, z * RCUT, 1e18, 1e21)).pvalue > 0.01, a
    assert np.array_equal(Z, np.select([A == 1, A == 4, A == 14, A == 56], [1, 2, 7, 26]))


def test_directions_isotropic_and_unit(oracle_lib):
    sp = O.spectrum(EQ1, 1.8, RCUT, 1e18, 1e21)
    n = 100000
    _, _, _, u, _ = O.source_sample(sp, 11, 0, n)
    assert np.max(np.abs(np.linalg.norm(u, axis=1) - 1.0)) < 4e-16
    assert np.all(np.abs(u.mean(0)) < 4.5 * math.sqrt(1 / 3 / n))
    assert stats.kstest(u[:, 2], "uniform", args=(-1, 2)).pvalue > 0.01
    phi = np.arctan2(u[:, 1], u[:, 0])
    assert stats.kstest(phi, "uniform", args=(-math.pi, 2 * math.pi)).pvalue > 0.01


def test_counter_based_reproducibility(oracle_lib):
    sp = O.spectrum(EQ1, 1.8, RCUT, 1e18, 1e21)
    full = O.source_sample(sp, 12, 0, 50)
    part = O.source_sample(sp, 12, 20, 30)
    for a, b in zip(full[:4], part[:4]):
        assert np.array_equal(a[20:], b)
    other = O.source_sample(sp, 13, 0, 50)
    assert not np.array_equal(full[2], other[2])


def test_invalid_spectra_rejected(oracle_lib):
    for sp in (O.spectrum([(1, 0, 1.0)], 1.8, RCUT, 1e18, 1e21),     # Z < 1
               O.spectrum([(1, 1, 1.0)], 1.8, RCUT, 1e21, 1e18),     # E_min > E_max
               O.spectrum([(1, 1, 0.0)], 1.8, RCUT, 1e18, 1e21),     # no weight
               O.spectrum([(1, 1, 1.0)], 1.8, -1.0, 1e18, 1e21)):    # cutoff <= 0
        with pytest.raises(ValueError):
            O.source_sample(sp, 1, 0, 3)


def test_cutoff_far_below_the_range_fails_loudly(oracle_lib):
    sp = O.spectrum([(1, 1, 1.0)], 1.8, 1e15, 1e19, 1e21)        # acceptance ~ exp(-1e4)
    A, _, _, _, failed = O.source_sample(sp, 1, 0, 5)
    assert failed == 5 and np.all(A == 0)


# ---- arrival map ---------------------------------------------------------------------------
def test_arrival_map_counts_finished_particles_above_threshold(oracle_lib):
    rng = np.random.default_rng(34)
    n, nside, thr = 3000, 8, 10 ** 18.7
    st = O.OracleState(n)
    st.c.n = n
    u = rng.standard_normal((n, 3))
    E = 10 ** rng.uniform(18, 20, n)
    status = rng.choice([O.DONE, O.ACTIVE, O.NAN], n, p=[0.8, 0.1, 0.1]).astype(np.int32)
    st.ux[:n], st.uy[:n], st.uz[:n] = u[:, 0], u[:, 1], u[:, 2]
    st.E[:n] = E
    st.status[:n] = status
    m = O.arrival_map(st, nside, thr)
    keep = (status == O.DONE) & (E > thr)
    ref = np.bincount(O.healpix_ring(nside, -u[keep]), minlength=12 * nside ** 2)
    assert np.array_equal(m, ref.astype(np.uint64)) and m.sum() == keep.sum()
