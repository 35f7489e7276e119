"""Lenses (paper Sec. 3.3) on the GPU against the oracle: one map within the FP64 summation
bound (lanes share a row, so the order of the additions differs), several maps bit for bit
(stored order), identity and permutation lenses exact, rigidity binning exact, and the full
nside-64, 24-bin synthetic lens checked on every row."""
import numpy as np
import pytest

import oracle as O
from paper_1410_5323_gb300 import inputs as I

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


def _bound(n_pix, rp, col, val, x):
    """Per row and map: 2 gamma_n sum |v x|, n the row's entries over all bins."""
    absx = np.abs(x)
    s = np.zeros((n_pix, x.shape[2]))
    for m in range(rp.shape[0]):
        r = rp[m]
        rows = np.repeat(np.arange(n_pix), np.diff(r))
        av = np.abs(val[r[0]:r[-1]]).astype(np.float64)
        for b in range(x.shape[2]):
            s[:, b] += np.bincount(rows, weights=av * absx[m][col[r[0]:r[-1]], b], minlength=n_pix)
    n = int(np.max(np.diff(rp, axis=1).sum(axis=0)))
    return 2 * (n * U / (1 - n * U)) * s


def _gpu(lens, x):
    import torch

    return lens.apply(torch.from_numpy(np.ascontiguousarray(x)).cuda()).cpu().numpy()


@pytest.mark.parametrize("k", [3, 12, 60])
def test_one_map_within_bound_every_group_size(oracle_lib, k):
    """Mean row lengths 3, 12, 60 pick 4, 16, 32 lanes per row."""
    import paper_1410_5323_gb300 as crp

    nside = 8
    n_pix = 12 * nside * nside
    rp, col, val = I.synthetic_lens(nside, I.lens_edges(5), seed=k, k=k)
    lens = crp.Lens(n_pix, rp, col, val)
    rng = np.random.default_rng(k)
    x = rng.standard_normal((5, n_pix)) * 10 ** rng.uniform(-3, 3, (5, n_pix))
    y = _gpu(lens, x)
    ref = O.lens_apply(n_pix, rp, col, val, x[:, :, None])[:, 0]
    assert np.all(np.abs(y - ref) <= _bound(n_pix, rp, col, val, x[:, :, None])[:, 0] + 1e-300)


@pytest.mark.parametrize("g", [4, 8, 16, 32])
def test_one_map_every_forced_group_size(oracle_lib, g):
    """The same lens with each group size forced: within the same bound."""
    import paper_1410_5323_gb300 as crp

    nside = 8
    n_pix = 12 * nside * nside
    rp, col, val = I.synthetic_lens(nside, I.lens_edges(5), seed=9, k=20)
    lens = crp.Lens(n_pix, rp, col, val)
    lens.set_group(g)
    x = np.random.default_rng(g).standard_normal((5, n_pix))
    y = _gpu(lens, x)
    ref = O.lens_apply(n_pix, rp, col, val, x[:, :, None])[:, 0]
    assert np.all(np.abs(y - ref) <= _bound(n_pix, rp, col, val, x[:, :, None])[:, 0] + 1e-300)


@pytest.mark.parametrize("n_maps", [2, 32, 45])
def test_several_maps_bit_identical(oracle_lib, n_maps):
    import paper_1410_5323_gb300 as crp

    nside = 8
    n_pix = 12 * nside * nside
    rp, col, val = I.synthetic_lens(nside, I.lens_edges(4), seed=5, k=20)
    lens = crp.Lens(n_pix, rp, col, val)
    x = np.random.default_rng(n_maps).standard_normal((4, n_pix, n_maps))
    assert np.array_equal(_gpu(lens, x), O.lens_apply(n_pix, rp, col, val, x))


def test_identity_and_permutation_exact(oracle_lib):
    import paper_1410_5323_gb300 as crp

    n_pix, n_mat = 3000, 3
    rng = np.random.default_rng(61)
    rp = np.stack([m * n_pix + np.arange(n_pix + 1) for m in range(n_mat)]).astype(np.int64)
    perms = [rng.permutation(n_pix) for _ in range(n_mat)]
    lens = crp.Lens(n_pix, rp, np.concatenate(perms), np.ones(n_mat * n_pix, np.float32))
    x = rng.integers(0, 10 ** 6, (n_mat, n_pix)).astype(np.float64)
    assert np.array_equal(_gpu(lens, x), sum(x[m][perms[m]] for m in range(n_mat)))


def test_empty_lens_and_invalid_lenses():
    import paper_1410_5323_gb300 as crp

    n_pix = 48
    lens = crp.Lens(n_pix, np.zeros((2, n_pix + 1), np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))
    assert np.all(_gpu(lens, np.ones((2, n_pix))) == 0.0)
    rp = np.zeros((1, n_pix + 1), np.int64)
    rp[0, 1:] = 1
    with pytest.raises(crp.CrpError):
        crp.Lens(n_pix, rp, np.array([n_pix], np.int32), np.ones(1, np.float32))     # column out of range
    rp[0, 5] = 0
    with pytest.raises(crp.CrpError):
        crp.Lens(n_pix, rp, np.array([0], np.int32), np.ones(1, np.float32))         # row_ptr decreases


def test_rigidity_binning_and_pipeline(oracle_lib):
    """Sampled Eq. 1 sources propagated a little, binned by rigidity on the GPU (exact counts),
    then lensed (within the bound)."""
    import paper_1410_5323_gb300 as crp

    nside = 8
    n_pix = 12 * nside * nside
    edges = I.lens_edges(6, 10 ** 18, 10 ** 21)
    rp, col, val = I.synthetic_lens(nside, edges, seed=7, k=16)
    lens = crp.Lens(n_pix, rp, col, val, edges)
    n = 5000
    g = I.kolmogorov_grid(16, 0.25 * I.MPC, 2, 8, 1e-13, 2).astype(np.float32)
    sim = crp.Simulation([crp.Field(g, 0.25 * I.MPC)], None, seed=4, capacity=n)
    sim.sample_sources(crp.Spectrum.of(I.EQ1_SPECIES, 1.8, 10 ** 19.8, 1e18, 1e21),
                       np.random.default_rng(62).uniform(0, 4 * I.MPC, (n, 3)))
    sim.propagate(1e-4, I.KPC, I.MPC, 10 * I.MPC, max_steps=80)
    assert sim.sync(timeout_s=300.0, raise_on_error=False) == 0
    xg = lens.bin(sim, nside, 10 ** 18.7).cpu().numpy()
    s = sim.state()
    st = O.OracleState(n)
    O.inject(st, I.Particles(np.stack([s["x"], s["y"], s["z"]], 1), np.stack([s["ux"], s["uy"], s["uz"]], 1),
                             s["E"], s["A"], s["Z"], s["uid"], s["grid_id"]), 4, None)
    st.status[:n] = s["status"]
    xo = O.lens_bin(st, nside, edges, 10 ** 18.7)
    assert np.array_equal(xg, xo) and xg.sum() > 0
    y = _gpu(lens, xg)
    ref = O.lens_apply(n_pix, rp, col, val, xo[:, :, None])[:, 0]
    assert np.all(np.abs(y - ref) <= _bound(n_pix, rp, col, val, xo[:, :, None])[:, 0])


def test_full_size_lens_every_row(oracle_lib):
    """nside 64 (49152 pixels), 24 rigidity bins, 24 entries per column: 28.3 M entries."""
    import paper_1410_5323_gb300 as crp

    nside = 64
    n_pix = 12 * nside * nside
    rp, col, val = I.synthetic_lens(nside, I.lens_edges(24), seed=1)
    lens = crp.Lens(n_pix, rp, col, val)
    x = np.random.default_rng(63).poisson(3.0, (24, n_pix)).astype(np.float64)
    y = _gpu(lens, x)
    ref = O.lens_apply(n_pix, rp, col, val, x[:, :, None])[:, 0]
    assert np.all(np.abs(y - ref) <= _bound(n_pix, rp, col, val, x[:, :, None])[:, 0])
    x32 = np.random.default_rng(64).poisson(3.0, (24, n_pix, 32)).astype(np.float64)
    assert np.array_equal(_gpu(lens, x32), O.lens_apply(n_pix, rp, col, val, x32))
