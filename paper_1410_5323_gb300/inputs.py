"""Seeded synthetic inputs for the 3D propagation workloads.

This module produces the *inputs* both the CUDA path and the CPU oracle consume:
turbulent field grids, interaction tables and injected particle batches. It holds
none of the propagation arithmetic (no stepping, lookup, interpolation or sampling
of interactions), so it can feed both sides without coupling them.

Paper passages the shapes follow (arXiv:1410.5323):
  * Sec. 4: vector field on a Cartesian grid initialised with a random turbulent
    realisation of a Kolmogorov power spectrum (coherence ~500 kpc, 50 kpc cells);
  * Sec. 4: sources emit isotropically with a power-law spectrum; the mixed
    composition uses H, He-4, N-14 and Fe-56;
  * Sec. 2: pair-production loss and photo-disintegration act on the nuclei; the
    paper's photon-background tables are not available, so closed-form synthetic
    tables with the same layout stand in for them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

MPC = 3.0856775814913673e22       # m  (648000/pi au, au = 149597870700 m)
KPC = MPC / 1000.0
NANOGAUSS = 1e-13                  # T

# Table geometry: x = log10(Lorentz factor) on [6, 14], 201 nodes, species (Z <= 26, N <= 30).
TABLE_Z_MAX = 26
TABLE_N_MAX = 30
TABLE_NODES = 201
TABLE_X0 = 6.0
TABLE_INV_DX = 25.0               # node spacing 0.04 in log10(gamma)

# Synthetic-table closed forms (constants are this project's readings).
LOSS_L0 = 1000.0 * MPC            # loss length scale of a proton at the break
LOSS_X_BREAK = 9.6                # log10 gamma of the loss-length minimum (node 90)
LOSS_SLOPE_LO = -3.0              # d log10(lambda)/d log10(gamma) below the break
LOSS_SLOPE_HI = 0.5               # ... above the break
PD_R0 = 1.0 / (5.0 * MPC)         # Fe-56 photo-disintegration rate on the plateau (1/m)
PD_X_THRESH = 9.0                 # log10 gamma where the plateau starts (node 75)
PD_SLOPE_LO = 2.0                 # d log10(R)/d log10(gamma) below it

SPECIES = {"H": (1, 1), "He": (4, 2), "N": (14, 7), "Fe": (56, 26)}


# --------------------------------------------------------------------------------------
# Kolmogorov turbulent field (Sec. 4)
# --------------------------------------------------------------------------------------
def _mode_integers(n: int) -> np.ndarray:
    return np.fft.fftfreq(n, d=1.0 / n)   # 0, 1, ..., n/2-1, -n/2, ..., -1


def kolmogorov_spectrum(n: int, lmin_cells: float, lmax_cells: float, seed: int) -> np.ndarray:
    """Complex mode amplitudes F[nx, ny, nz, 3] of one Kolmogorov realisation (unscaled).

    Active modes: integer wavevectors with n/lmax <= |k| <= n/lmin and no component on a
    Nyquist plane (|k_i| = n/2). Each active mode gets amplitude |k|^(-11/6) (per-mode power
    |k|^(-11/3), shell power |k|^(-5/3)), a random unit polarisation perpendicular to k (so
    the field is divergence-free) and a uniform random phase. The spectrum is made Hermitian
    (F(-k) = conj F(k)) so that the inverse FFT is real.
    """
    if n % 2:
        raise ValueError("grid size must be even")
    rng = np.random.Generator(np.random.PCG64(seed))
    k1 = _mode_integers(n)
    kx, ky, kz = np.meshgrid(k1, k1, k1, indexing="ij")
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    nyq = -(n // 2)
    active = (kk >= n / lmax_cells) & (kk <= n / lmin_cells)
    active &= (kx != nyq) & (ky != nyq) & (kz != nyq)
    # random polarisation, projected perpendicular to k
    e = rng.standard_normal((n, n, n, 3))
    phase = rng.uniform(0.0, 2.0 * np.pi, (n, n, n))
    safe = np.where(kk > 0, kk, 1.0)
    khat = np.stack([kx / safe, ky / safe, kz / safe], axis=-1)
    e = e - np.sum(e * khat, axis=-1, keepdims=True) * khat
    enorm = np.linalg.norm(e, axis=-1, keepdims=True)
    e = e / np.where(enorm > 0, enorm, 1.0)
    amp = np.where(active, safe ** (-11.0 / 6.0), 0.0)
    F = (amp * np.exp(1j * phase))[..., None] * e
    # Hermitian symmetry: keep the "positive" half, mirror the other
    pos = (kx > 0) | ((kx == 0) & (ky > 0)) | ((kx == 0) & (ky == 0) & (kz > 0))
    mirror = np.roll(np.flip(F, axis=(0, 1, 2)), 1, axis=(0, 1, 2))   # F[(-i) mod n]
    F = np.where(pos[..., None], F, np.conj(mirror))
    return F


def kolmogorov_grid(n: int, spacing_m: float, lmin_cells: float, lmax_cells: float,
                    brms_t: float, seed: int) -> np.ndarray:
    """Real periodic field B[nx, ny, nz, 3] (tesla, float64) with <|B|^2> = brms^2."""
    F = kolmogorov_spectrum(n, lmin_cells, lmax_cells, seed)
    B = np.empty((n, n, n, 3), dtype=np.float64)
    for c in range(3):
        B[..., c] = np.fft.ifftn(F[..., c]).real
    del F
    rms = math.sqrt(float(np.mean(np.sum(B * B, axis=-1))))
    B *= brms_t / rms
    return B


def kolmogorov_grid_torch(n: int, lmin_cells: float, lmax_cells: float, brms_t: float,
                          seed: int, device: str = "cuda"):
    """Same recipe as :func:`kolmogorov_grid`, built with torch one component at a time
    (for grids too large for host FFTs, e.g. 1024^3 on the GPU). FP32 spectrum and FFT.

    Randomness comes from a seeded torch generator on that device, so the realisation
    differs from the numpy one for the same seed but is reproducible on one machine.
    Returns B [n, n, n, 3] float32 (tesla) with <|B|^2> = brms^2.
    """
    import torch

    if n % 2:
        raise ValueError("grid size must be even")
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    k1 = torch.fft.fftfreq(n, d=1.0 / n, device=device, dtype=torch.float32)
    kx, ky, kz = k1.view(n, 1, 1), k1.view(1, n, 1), k1.view(1, 1, n)
    kk = torch.sqrt(kx * kx + ky * ky + kz * kz)
    nyq = -(n // 2)
    active = (kk >= n / lmax_cells) & (kk <= n / lmin_cells)
    active &= (kx != nyq) & (ky != nyq) & (kz != nyq)
    safe = torch.where(kk > 0, kk, torch.ones_like(kk))
    # random polarisation perpendicular to k, unit length, times |k|^(-11/6)
    e = torch.randn((3, n, n, n), generator=g, device=device, dtype=torch.float32)
    phase = torch.rand((n, n, n), generator=g, device=device, dtype=torch.float32) * (2 * math.pi)
    kh = (kx / safe, ky / safe, kz / safe)
    dot = e[0] * kh[0] + e[1] * kh[1] + e[2] * kh[2]
    for c in range(3):
        e[c] -= dot * kh[c]
    del dot
    en = torch.sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2])
    amp = torch.where(active, safe ** (-11.0 / 6.0) / torch.where(en > 0, en, torch.ones_like(en)),
                      torch.zeros_like(safe))
    del en, kk, safe, active
    pos = (kx > 0) | ((kx == 0) & (ky > 0)) | ((kx == 0) & (ky == 0) & (kz > 0))
    cos_p, sin_p = torch.cos(phase), torch.sin(phase)
    del phase
    out = torch.empty((n, n, n, 3), dtype=torch.float32, device=device)
    sumsq = 0.0
    for c in range(3):
        a = amp * e[c]
        Fc = torch.complex(a * cos_p, a * sin_p)
        del a
        mirror = torch.roll(torch.flip(Fc, dims=(0, 1, 2)), shifts=(1, 1, 1), dims=(0, 1, 2))
        Fc = torch.where(pos, Fc, torch.conj(mirror))
        del mirror
        Bc = torch.fft.ifftn(Fc).real
        del Fc
        sumsq += float(torch.sum(Bc.double() ** 2))
        out[..., c] = Bc
        del Bc
    out *= float(brms_t / math.sqrt(sumsq / n ** 3))
    return out


# --------------------------------------------------------------------------------------
# Modulation grid (Sec. 3.2 modulated grids; Sec. 4 scenario: density -> field strength)
# --------------------------------------------------------------------------------------
def _band_filter(k, n: int, lmin_cells: float, lmax_cells: float, slope: float):
    """|k|^slope on the band n/lmax <= |k| <= n/lmin, zero elsewhere (and at k = 0)."""
    safe = np.where(k > 0, k, 1.0)
    return np.where((k >= n / lmax_cells) & (k <= n / lmin_cells), safe ** slope, 0.0)


def density_field(n: int, lmin_cells: float, lmax_cells: float, sigma_ln: float,
                  seed: int) -> np.ndarray:
    """Log-normal matter density rho [n, n, n] (float64, mean 1), periodic.

    A Gaussian random field G with power |k|^-2 on the band n/lmax <= |k| <= n/lmin (white
    noise filtered by |k|^-1, real FFTs), scaled to unit variance; rho = exp(sigma G -
    sigma^2/2), renormalised to mean 1. A synthetic stand-in for a constrained large-scale
    structure simulation: voids to clusters over exp(+-3 sigma)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    white = rng.standard_normal((n, n, n))
    F = np.fft.rfftn(white)
    del white
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    kz = np.fft.rfftfreq(n, d=1.0 / n)
    k = np.sqrt(k1[:, None, None] ** 2 + k1[None, :, None] ** 2 + kz[None, None, :] ** 2)
    F *= _band_filter(k, n, lmin_cells, lmax_cells, -1.0)
    del k
    G = np.fft.irfftn(F, s=(n, n, n), axes=(0, 1, 2))
    del F
    G /= G.std()
    rho = np.exp(sigma_ln * G - 0.5 * sigma_ln * sigma_ln)
    rho /= rho.mean()
    return rho


def modulation_from_density(rho, exponent: float = 2.0 / 3.0) -> np.ndarray:
    """Field-strength modulation M = rho^exponent (flux freezing under isotropic
    compression: B ~ rho^(2/3)), normalised to <M^2> = 1 so that the modulated field keeps
    the vector grid's B_rms on average. float32 [n, n, n]."""
    M = np.power(rho, exponent)
    M /= math.sqrt(float(np.mean(M * M)))
    return M.astype(np.float32)


def density_positions(n_particles: int, rho: np.ndarray, spacing_m: float, seed: int,
                      origin_m=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Source positions [n, 3] (m) distributed like the matter density: a cell drawn with
    probability proportional to rho, then a uniform point inside it."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    cdf = np.cumsum(rho.ravel(), dtype=np.float64)
    cells = np.searchsorted(cdf, rng.uniform(0.0, cdf[-1], n_particles), side="right")
    cells = np.minimum(cells, rho.size - 1)
    ijk = np.stack(np.unravel_index(cells, rho.shape), axis=1).astype(np.float64)
    return np.asarray(origin_m) + (ijk + rng.uniform(0.0, 1.0, (n_particles, 3))) * spacing_m


def quantize_bf16(B, scale: float | None = None):
    """BF16 storage with one FP32 scale: B ~= scale * stored. Returns (stored bfloat16 tensor,
    scale as a Python float that is exactly an FP32 value). Default scale: the rms of |B|."""
    import torch

    if scale is None:
        scale = float(torch.sqrt(torch.mean(torch.sum(B.double() ** 2, dim=-1))))
    scale = float(np.float32(scale))
    return (B * (1.0 / scale)).to(torch.bfloat16), scale


# --------------------------------------------------------------------------------------
# Synthetic interaction tables (Sec. 2 processes; closed forms are readings)
# --------------------------------------------------------------------------------------
@dataclasses.dataclass
class TableArrays:
    z_max: int
    n_max: int
    n_nodes: int
    x0: float
    inv_dx: float
    log10_loss: np.ndarray     # [species, n_nodes] float64, log10 of 1/lambda_loss (1/m)
    log10_pd: np.ndarray       # [species, n_nodes] float64, log10 of the PD rate (1/m)
    has_loss: np.ndarray       # [species] uint8
    has_pd: np.ndarray         # [species] uint8

    def species_index(self, A: int, Z: int) -> int:
        return Z * (self.n_max + 1) + (A - Z)


def table_nodes(n_nodes: int = TABLE_NODES, x0: float = TABLE_X0, inv_dx: float = TABLE_INV_DX):
    return x0 + np.arange(n_nodes, dtype=np.float64) / inv_dx


def loss_rate_closed_form(A, Z, x):
    """1/lambda_loss (1/m) at log10 gamma = x: a broken power law in gamma with its break
    at 10^9.6; lambda scales as A/Z^2 times 1000 Mpc at the break."""
    A = np.asarray(A, dtype=np.float64)
    Z = np.asarray(Z, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    slope = np.where(x < LOSS_X_BREAK, LOSS_SLOPE_LO, LOSS_SLOPE_HI)
    lam = (A / (Z * Z)) * LOSS_L0 * np.power(10.0, slope * (x - LOSS_X_BREAK))
    return 1.0 / lam


def pd_rate_closed_form(A, x):
    """Photo-disintegration rate (1/m): R0 (A/56) (gamma/10^9)^2 below 10^9, flat above."""
    A = np.asarray(A, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    return PD_R0 * (A / 56.0) * np.power(10.0, PD_SLOPE_LO * np.minimum(x - PD_X_THRESH, 0.0))


def synthetic_tables(z_max: int = TABLE_Z_MAX, n_max: int = TABLE_N_MAX,
                     n_nodes: int = TABLE_NODES, x0: float = TABLE_X0,
                     inv_dx: float = TABLE_INV_DX) -> TableArrays:
    x = table_nodes(n_nodes, x0, inv_dx)
    n_sp = (z_max + 1) * (n_max + 1)
    ll = np.full((n_sp, n_nodes), -np.inf)
    lp = np.full((n_sp, n_nodes), -np.inf)
    hl = np.zeros(n_sp, dtype=np.uint8)
    hp = np.zeros(n_sp, dtype=np.uint8)
    for Z in range(z_max + 1):
        for N in range(n_max + 1):
            A = Z + N
            sp = Z * (n_max + 1) + N
            if A < 1:
                continue
            if Z > 0:
                # log10 of the closed form, written as the linear function of x it is
                slope = np.where(x < LOSS_X_BREAK, LOSS_SLOPE_LO, LOSS_SLOPE_HI)
                ll[sp] = -(math.log10(A / (Z * Z) * LOSS_L0) + slope * (x - LOSS_X_BREAK))
                hl[sp] = 1
            if A > 1:
                lp[sp] = math.log10(PD_R0 * A / 56.0) + PD_SLOPE_LO * np.minimum(x - PD_X_THRESH, 0.0)
                hp[sp] = 1
    return TableArrays(z_max, n_max, n_nodes, x0, inv_dx, ll, lp, hl, hp)


def constant_rate_tables(loss_rate: float = 0.0, pd_rate: float = 0.0,
                         z_max: int = TABLE_Z_MAX, n_max: int = TABLE_N_MAX) -> TableArrays:
    """Tables with the same rate at every gamma (for closed-form checks: E(s) = E0 exp(-s R),
    Poisson interaction counts)."""
    n_sp = (z_max + 1) * (n_max + 1)
    ll = np.full((n_sp, TABLE_NODES), -np.inf)
    lp = np.full((n_sp, TABLE_NODES), -np.inf)
    hl = np.zeros(n_sp, dtype=np.uint8)
    hp = np.zeros(n_sp, dtype=np.uint8)
    for Z in range(z_max + 1):
        for N in range(n_max + 1):
            A = Z + N
            sp = Z * (n_max + 1) + N
            if A < 1:
                continue
            if loss_rate > 0 and Z > 0:
                ll[sp] = math.log10(loss_rate)
                hl[sp] = 1
            if pd_rate > 0 and A > 1:
                lp[sp] = math.log10(pd_rate)
                hp[sp] = 1
    return TableArrays(z_max, n_max, TABLE_NODES, TABLE_X0, TABLE_INV_DX, ll, lp, hl, hp)


# --------------------------------------------------------------------------------------
# Particle batches (Sec. 4: isotropic point emission, power-law spectra)
# --------------------------------------------------------------------------------------
@dataclasses.dataclass
class Particles:
    x: np.ndarray      # [n, 3] float64, m
    u: np.ndarray      # [n, 3] float64, unit direction
    E: np.ndarray      # [n] float64, eV
    A: np.ndarray      # [n] int32
    Z: np.ndarray      # [n] int32
    uid: np.ndarray    # [n] int64, < 2^32
    grid_id: np.ndarray  # [n] int32

    def __len__(self):
        return int(self.E.shape[0])

    def take(self, idx) -> "Particles":
        return Particles(self.x[idx].copy(), self.u[idx].copy(), self.E[idx].copy(),
                         self.A[idx].copy(), self.Z[idx].copy(), self.uid[idx].copy(),
                         self.grid_id[idx].copy())


def isotropic_directions(n: int, rng: np.random.Generator) -> np.ndarray:
    w = rng.uniform(-1.0, 1.0, n)
    phi = rng.uniform(0.0, 2.0 * np.pi, n)
    sw = np.sqrt(1.0 - w * w)
    return np.stack([sw * np.cos(phi), sw * np.sin(phi), w], axis=1)


def power_law_energies(n: int, rng, e_min: float, e_max: float, index: float) -> np.ndarray:
    """dN/dE ~ E^-index on [e_min, e_max] by inverse CDF (index != 1)."""
    u = rng.uniform(0.0, 1.0, n)
    g = 1.0 - index
    return (e_min ** g + u * (e_max ** g - e_min ** g)) ** (1.0 / g)


def log_uniform_energies(n: int, rng, e_min: float, e_max: float) -> np.ndarray:
    return np.exp(rng.uniform(math.log(e_min), math.log(e_max), n))


def make_particles(n: int, seed: int, species=(("H", 1.0),), energy=("fixed", 1e19),
                   grid_ids=None, uid_offset: int = 0) -> Particles:
    """Isotropic emission from the origin. ``species``: (name, fraction) pairs, drawn
    by fraction; ``energy``: ("fixed", E) | ("power", e_min, e_max, index) |
    ("loguniform", e_min, e_max)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    names = [s for s, _ in species]
    frac = np.array([f for _, f in species], dtype=np.float64)
    frac = frac / frac.sum()
    pick = rng.choice(len(names), size=n, p=frac) if len(names) > 1 else np.zeros(n, dtype=np.int64)
    A = np.array([SPECIES[names[i]][0] for i in range(len(names))], dtype=np.int32)[pick]
    Z = np.array([SPECIES[names[i]][1] for i in range(len(names))], dtype=np.int32)[pick]
    kind = energy[0]
    if kind == "fixed":
        E = np.full(n, float(energy[1]))
    elif kind == "power":
        E = power_law_energies(n, rng, energy[1], energy[2], energy[3])
    elif kind == "loguniform":
        E = log_uniform_energies(n, rng, energy[1], energy[2])
    else:
        raise ValueError(kind)
    u = isotropic_directions(n, rng)
    x = np.zeros((n, 3))
    uid = np.arange(n, dtype=np.int64) + uid_offset
    gid = np.zeros(n, dtype=np.int32) if grid_ids is None else np.asarray(grid_ids, dtype=np.int32)
    return Particles(x, u, E, A, Z, uid, gid)


# --------------------------------------------------------------------------------------
# Workloads (sizes and parameters; synthetic stand-ins for the paper's Sec. 4 scenario)
# --------------------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    name: str
    n_particles: int
    grid_n: int
    spacing_m: float
    lmin_cells: float
    lmax_cells: float
    brms_t: float
    grid_seed: int
    tol: float
    hmin_m: float
    hmax_m: float
    dmax_m: float
    species: tuple
    energy: tuple
    interactions: bool
    n_grids: int = 1
    particle_seed: int = 1
    rng_seed: int = 1          # Philox key for interaction sampling
    # modulation grid (modulated workloads only): n^3 cells of mod_spacing_m, density with
    # log-normal width mod_sigma_ln on mod_lmin..mod_lmax cells, sources follow the density
    mod_n: int = 0
    mod_spacing_m: float = 0.0
    mod_lmin_cells: float = 2.0
    mod_lmax_cells: float = 0.0
    mod_sigma_ln: float = 0.0
    mod_seed: int = 2
    reflect: bool = False      # reflective box = the modulation grid's volume
    # sources drawn on the device from Eq. 1: ((A, Z, x), ...), alpha, R_cut (V), E range (eV)
    spectrum: tuple | None = None
    arrival_nside: int = 0     # arrival map resolution (0: none) and its energy threshold
    arrival_emin_ev: float = 0.0
    bf16: bool = False         # grid generated on the device (torch FFT) and stored as BF16 + scale


EQ1_SPECIES = ((1, 1, 1.0), (4, 2, 0.5), (14, 7, 0.3), (56, 26, 0.1))   # Sec. 4: H, He, N, Fe
EQ1_SPECTRUM = (EQ1_SPECIES, 1.8, 10 ** 19.8, 1e18, 1e21)


def workload_box(w: Workload):
    """(origin[3], size[3]) of the workload's reflective box in metres, or None."""
    if not w.reflect:
        return None
    L = w.mod_n * w.mod_spacing_m
    return (0.0, 0.0, 0.0), (L, L, L)


def workload(name: str) -> Workload:
    """The synthetic workloads (turbulent grid, injection, propagation limits)."""
    common = dict(spacing_m=0.25 * MPC, lmin_cells=2.0, tol=1e-4, hmin_m=1.0 * KPC,
                  hmax_m=1.0 * MPC, grid_seed=1)
    if name == "fp64_64cube_1k_protons":
        return Workload(name, 1024, 64, lmax_cells=32.0, brms_t=1.0 * NANOGAUSS,
                        dmax_m=100.0 * MPC, species=(("H", 1.0),), energy=("fixed", 1e19),
                        interactions=False, **common)
    if name == "fp64_256cube_1M_nuclei":
        return Workload(name, 1_000_000, 256, lmax_cells=32.0, brms_t=1.0 * NANOGAUSS,
                        dmax_m=500.0 * MPC,
                        species=(("H", 0.4), ("He", 0.3), ("N", 0.2), ("Fe", 0.1)),
                        energy=("power", 1e18, 10 ** 20.5, 2.0), interactions=True, **common)
    if name == "mixed_1024cube_10M_pFe":
        return Workload(name, 10_000_000, 1024, lmax_cells=256.0, brms_t=0.5 * NANOGAUSS,
                        dmax_m=500.0 * MPC, species=(("H", 0.5), ("Fe", 0.5)),
                        energy=("power", 1e18, 10 ** 20.5, 2.0), interactions=False, bf16=True, **common)
    if name == "batched_64x128cube_12.8M_protons":
        return Workload(name, 64 * 200_000, 128, lmax_cells=32.0, brms_t=1.0 * NANOGAUSS,
                        dmax_m=100.0 * MPC, species=(("H", 1.0),),
                        energy=("loguniform", 1e17, 10 ** 20.5), interactions=False,
                        n_grids=64, **common)
    if name == "modulated_440cube_300kpc_x_256cube_50kpc_1M_nuclei":
        # Sec. 4 geometry: modulation 132 Mpc at 300 kpc; vector grid at 50 kpc with a 500 kpc
        # coherence length (Kolmogorov on 100 kpc .. 2.2 Mpc)
        return Workload(name, 1_000_000, 256, spacing_m=50.0 * KPC, lmin_cells=2.0,
                        lmax_cells=44.0, brms_t=1.0 * NANOGAUSS, grid_seed=1, tol=1e-4,
                        hmin_m=1.0 * KPC, hmax_m=1.0 * MPC, dmax_m=100.0 * MPC,
                        species=(("H", 0.4), ("He", 0.3), ("N", 0.2), ("Fe", 0.1)),
                        energy=("power", 1e18, 10 ** 20.5, 2.0), interactions=True,
                        mod_n=440, mod_spacing_m=300.0 * KPC, mod_lmin_cells=2.0,
                        mod_lmax_cells=110.0, mod_sigma_ln=1.0, reflect=True)
    if name == "sec4_eq1_440cube_x_256cube_1M_nuclei":
        # the full Sec. 4 scenario: modulated field and reflective box as above, sources at
        # density-weighted positions drawn from Eq. 1 on the device, arrival map (HEALPix
        # nside 64) of events above 10^18.7 eV
        w = workload("modulated_440cube_300kpc_x_256cube_50kpc_1M_nuclei")
        w.name = name
        w.spectrum = EQ1_SPECTRUM
        w.species = tuple((str(a), x) for a, _, x in EQ1_SPECIES)   # informational
        w.energy = ("eq1",)
        w.arrival_nside = 64
        w.arrival_emin_ev = 10 ** 18.7
        return w
    if name == "adjoint_128cube_4k_protons":
        return Workload(name, 4096, 128, lmax_cells=32.0, brms_t=1.0 * NANOGAUSS,
                        dmax_m=1e6 * MPC, species=(("H", 1.0),), energy=("fixed", 10 ** 19.5),
                        interactions=False, **common)
    raise KeyError(name)


def batched_brms(n_grids: int = 64, seed: int = 1, lo: float = 0.1, hi: float = 10.0) -> np.ndarray:
    """Per-realisation B_rms (tesla), log-uniform in [lo, hi] nG."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    return np.exp(rng.uniform(math.log(lo), math.log(hi), n_grids)) * NANOGAUSS


def batched_grids(w: Workload, n_grids: int | None = None, grid_n: int | None = None, ids=None):
    """Field realisations of the batching workload: seeds 1..n, B_rms log-uniform in
    [0.1, 10] nG, each an FP32 [n, n, n, 3] Kolmogorov grid. With `ids`, only those
    realisations (same seeds and B_rms as in the whole set)."""
    n_grids = n_grids or w.n_grids
    grid_n = grid_n or w.grid_n
    brms = batched_brms(n_grids)
    ids = range(n_grids) if ids is None else [int(i) for i in ids]
    return [kolmogorov_grid(grid_n, w.spacing_m, w.lmin_cells, w.lmax_cells, float(brms[i]),
                            i + 1).astype(np.float32) for i in ids], brms


def batched_particles(w: Workload, n_per_grid: int, n_grids: int | None = None, seed: int = 1):
    """Protons, log-uniform energies, n_per_grid per realisation (grid_id = i // n_per_grid)."""
    n_grids = n_grids or w.n_grids
    n = n_per_grid * n_grids
    gid = np.repeat(np.arange(n_grids, dtype=np.int32), n_per_grid)
    return make_particles(n, seed, w.species, w.energy, grid_ids=gid)


# --------------------------------------------------------------------------------------
# Synthetic lenses (Sec. 3.3: per-rigidity transfer matrices over HEALPix pixels)
# --------------------------------------------------------------------------------------
def healpix_centres(nside: int) -> np.ndarray:
    """Unit vectors [12 nside^2, 3] of the HEALPix RING pixel centres (Gorski et al. 2005):
    cap rings i < nside at z = 1 - i^2/(3 nside^2), phi = pi/(2i) (j + 1/2); belt rings at
    z = 4/3 - 2i/(3 nside), phi = pi/(2 nside) (j + s/2), s = (i - nside + 1) mod 2."""
    zs, ph = [], []
    for i in range(1, nside):
        j = np.arange(4 * i)
        zs.append(np.full(4 * i, 1.0 - i * i / (3.0 * nside * nside)))
        ph.append(math.pi / (2 * i) * (j + 0.5))
    for i in range(nside, 3 * nside + 1):
        j = np.arange(4 * nside)
        zs.append(np.full(4 * nside, 4.0 / 3.0 - 2.0 * i / (3.0 * nside)))
        ph.append(math.pi / (2 * nside) * (j + ((i - nside + 1) % 2) / 2.0))
    for i in range(nside - 1, 0, -1):
        j = np.arange(4 * i)
        zs.append(np.full(4 * i, -(1.0 - i * i / (3.0 * nside * nside))))
        ph.append(math.pi / (2 * i) * (j + 0.5))
    z = np.concatenate(zs)
    phi = np.concatenate(ph)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)


def lens_edges(n_mat: int, r_min_v: float = 10 ** 18.5, r_max_v: float = 10 ** 21.0) -> np.ndarray:
    """Rigidity bin edges (V), log-spaced."""
    return np.logspace(math.log10(r_min_v), math.log10(r_max_v), n_mat + 1)


def synthetic_lens(nside: int, edges, seed: int = 1, k: int = 24):
    """A synthetic lens standing in for galactic-field lenses built by backtracking: for each
    rigidity bin (centre R) and border pixel s, the arrival directions are spread around the
    border direction rotated by delta(R) = 30 deg (10^19 V / R) (capped at 90 deg) about a
    fixed random axis, with a Gaussian profile of width sigma(R) = max(0.5 deg,
    3 deg (10^19 V / R)); the k pixels nearest to that centre carry the column, weights
    normalised to a transmission 1 - 0.3 exp(-R / 10^19 V). k = 24 keeps a nside-64 matrix at
    9.4 MB, inside the "less than 10 MB per matrix" of Sec. 3.3. Returns (row_ptr [n_mat, n_pix+1]
    int64 with offsets into col/val, col int32, val float32) in CSR form, rows = arrival pixels."""
    from scipy.spatial import cKDTree

    rng = np.random.Generator(np.random.PCG64(seed))
    c = healpix_centres(nside)
    n_pix = len(c)
    tree = cKDTree(c)
    axis = rng.standard_normal(3)
    axis /= np.linalg.norm(axis)
    edges = np.asarray(edges, dtype=np.float64)
    row_ptr = np.zeros((len(edges) - 1, n_pix + 1), dtype=np.int64)
    cols, vals = [], []
    offset = 0
    for m in range(len(edges) - 1):
        R = math.sqrt(edges[m] * edges[m + 1])
        delta = math.radians(min(90.0, 30.0 * 1e19 / R))
        sigma = math.radians(max(0.5, 3.0 * 1e19 / R))
        # Rodrigues rotation of every centre about `axis` by delta
        cd, sd = math.cos(delta), math.sin(delta)
        rot = c * cd + np.cross(axis, c) * sd + np.outer(c @ axis, axis) * (1 - cd)
        d, idx = tree.query(rot, k=k)                  # chord distances, [n_pix, k]
        ang = 2.0 * np.arcsin(np.minimum(1.0, d / 2.0))
        w = np.exp(-0.5 * (ang / sigma) ** 2)
        w *= (1.0 - 0.3 * math.exp(-R / 1e19)) / w.sum(axis=1, keepdims=True)
        # CSR with rows = arrival pixel (idx), columns = border pixel s
        rows = idx.ravel()
        colsm = np.repeat(np.arange(n_pix, dtype=np.int64), k)
        order = np.lexsort((colsm, rows))
        rows, colsm, wv = rows[order], colsm[order], w.ravel()[order]
        counts = np.bincount(rows, minlength=n_pix)
        row_ptr[m, 1:] = offset + np.cumsum(counts)
        row_ptr[m, 0] = offset
        cols.append(colsm.astype(np.int32))
        vals.append(wv.astype(np.float32))
        offset += len(rows)
    return row_ptr, np.concatenate(cols), np.concatenate(vals)

