"""Pins of the oracle's lens (Sec. 3.3): per-rigidity sparse matrices applied to arrival maps
and the rigidity-binned maps they take. References: scipy.sparse products within the FP64
summation bound, identity and permutation lenses (exact on integer maps), linearity in the
maps, brute-force binning."""
import numpy as np
import pytest
import scipy.sparse as sps

import oracle as O
from paper_1410_5323_gb300 import inputs as I

U = 2.0 ** -53


def _scipy_mats(n_pix, rp, col, val):
    return [sps.csr_matrix((val[rp[m, 0]:rp[m, -1]].astype(np.float64), col[rp[m, 0]:rp[m, -1]],
                            rp[m] - rp[m, 0]), shape=(n_pix, n_pix)) for m in range(rp.shape[0])]


def _bound(n_pix, rp, col, val, x):
    """2 gamma_n sum |v x| per row and map: the FP64 error bound of any summation order, for
    the oracle and for scipy, so their difference stays below twice of it."""
    mats = _scipy_mats(n_pix, rp, col, val)
    absx = np.abs(x)
    s = sum(abs(M) @ absx[m] for m, M in enumerate(mats))
    n = np.max(np.diff(rp, axis=1).sum(axis=0))
    g = n * U / (1 - n * U)
    return 2 * g * s


@pytest.fixture(scope="module")
def lens8():
    nside = 8
    edges = I.lens_edges(5)
    rp, col, val = I.synthetic_lens(nside, edges, seed=3, k=8)
    return nside, 12 * nside * nside, edges, rp, col, val


def test_matches_scipy_within_the_summation_bound(oracle_lib, lens8):
    _, n_pix, _, rp, col, val = lens8
    rng = np.random.default_rng(41)
    x = rng.standard_normal((rp.shape[0], n_pix, 3)) * 10 ** rng.uniform(-3, 3, (rp.shape[0], n_pix, 1))
    y = O.lens_apply(n_pix, rp, col, val, x)
    mats = _scipy_mats(n_pix, rp, col, val)
    ref = sum(M @ x[m] for m, M in enumerate(mats))
    assert np.all(np.abs(y - ref) <= _bound(n_pix, rp, col, val, x) + 1e-300)


def test_maps_are_independent_and_linear(oracle_lib, lens8):
    _, n_pix, _, rp, col, val = lens8
    rng = np.random.default_rng(42)
    x = rng.integers(0, 50, (rp.shape[0], n_pix, 4)).astype(np.float64)
    y = O.lens_apply(n_pix, rp, col, val, x)
    for b in range(4):
        assert np.array_equal(y[:, b], O.lens_apply(n_pix, rp, col, val, x[:, :, b:b + 1])[:, 0])


def test_identity_and_permutation_lenses_exact(oracle_lib):
    n_pix, n_mat = 300, 4
    rng = np.random.default_rng(43)
    x = rng.integers(0, 1000, (n_mat, n_pix, 2)).astype(np.float64)
    # identity in every bin
    rp = np.stack([m * n_pix + np.arange(n_pix + 1) for m in range(n_mat)]).astype(np.int64)
    col = np.tile(np.arange(n_pix), n_mat).astype(np.int32)
    val = np.ones(n_mat * n_pix, np.float32)
    assert np.array_equal(O.lens_apply(n_pix, rp, col, val, x), x.sum(axis=0))
    # a permutation per bin: row p takes column perm[m][p]
    perms = [rng.permutation(n_pix) for _ in range(n_mat)]
    col = np.concatenate(perms).astype(np.int32)
    ref = sum(x[m][perms[m]] for m in range(n_mat))
    assert np.array_equal(O.lens_apply(n_pix, rp, col, val, x), ref)


def test_transmission_is_the_column_sum(oracle_lib, lens8):
    """A map with one count in border pixel s gives the column s of each matrix; its total is
    that bin's transmission 1 - 0.3 exp(-R/10^19 V) (to FP32 rounding of the weights)."""
    _, n_pix, edges, rp, col, val = lens8
    for m in range(rp.shape[0]):
        x = np.zeros((rp.shape[0], n_pix, 1))
        x[m, 17, 0] = 1.0
        y = O.lens_apply(n_pix, rp, col, val, x)
        R = np.sqrt(edges[m] * edges[m + 1])
        assert abs(y.sum() - (1 - 0.3 * np.exp(-R / 1e19))) < 1e-6


def test_empty_lens_gives_zero(oracle_lib):
    n_pix = 48
    rp = np.zeros((2, n_pix + 1), np.int64)
    y = O.lens_apply(n_pix, rp, np.zeros(0, np.int32), np.zeros(0, np.float32), np.ones((2, n_pix, 1)))
    assert np.all(y == 0.0)


def test_rigidity_binning_brute_force(oracle_lib):
    rng = np.random.default_rng(44)
    n, nside = 5000, 4
    edges = I.lens_edges(6)
    st = O.OracleState(n)
    st.c.n = n
    u = rng.standard_normal((n, 3))
    Z = rng.choice([-1, 0, 1, 2, 26], n).astype(np.int32)
    E = 10 ** rng.uniform(18, 22.5, n)
    status = rng.choice([O.DONE, O.ACTIVE], n, p=[0.85, 0.15]).astype(np.int32)
    st.ux[:n], st.uy[:n], st.uz[:n] = u[:, 0], u[:, 1], u[:, 2]
    st.E[:n], st.Z[:n], st.status[:n] = E, Z, status
    x = O.lens_bin(st, nside, edges, 10 ** 18.7)
    ref = np.zeros_like(x)
    for i in range(n):
        if status[i] != O.DONE or Z[i] <= 0 or not E[i] > 10 ** 18.7:
            continue
        R = E[i] / Z[i]
        m = np.searchsorted(edges, R, side="right") - 1
        if 0 <= m < len(edges) - 1:
            ref[m, O.healpix_ring(nside, -u[i:i + 1])[0]] += 1
    assert np.array_equal(x, ref) and 0 < x.sum() < n
