"""Pins of the oracle's interaction modules (paper Sec. 2: pair-production loss,
photo-disintegration with nucleon secondaries) and of its bookkeeping."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle as O
from paper_1410_5323_gb300 import inputs as I
from _oracle_helpers import particles, run, uniform_grid

MP = 938272088.16


def _by_uid(st):
    snap = st.snapshot()
    order = np.argsort(snap["uid"], kind="stable")
    return {k: v[order] for k, v in snap.items()}


def _f32_rate_bound(rate, E=1e21, slope=3.0):
    """Relative error bound of the FP32 rate evaluation (u = 2^-24 per rounding):
    exponent y = v log2 10: two roundings of |y| -> ln2 u (2|y| + 2);
    the FP32 table entries and interpolation: ln10 u 2|v|;
    the coordinate x = log10 gamma0: log2 E and log2(A m_p c^2) (< 90 each), their difference
    and the scaling, plus the 23-bit truncation of each argument (2 x 1.7e-7), times the
    table's slope d log10 rate / d log10 gamma (<= 3 here), times ln10."""
    u = 2.0 ** -24
    y = abs(math.log2(rate))
    v = abs(math.log10(rate))
    lgE = abs(math.log2(E))
    x_err = (u * (lgE + 90.0 + 90.0 + 4.0) + 2 * 1.72e-7) * math.log10(2.0)
    return math.log(2.0) * u * (2 * y + 2) + math.log(10.0) * (u * 2 * v + slope * x_err)


def test_table_interpolation_reproduces_closed_form(oracle_lib):
    """Breaks sit on nodes and log10 rates are linear in log10(gamma) between them, so the
    log-linear interpolation equals the closed form; the FP32 evaluation stays within its
    stated bound (a pure relative tolerance: the rates are ~1e-25 per metre)."""
    t = I.synthetic_tables()
    ot = O.OracleTables(t)
    rng = np.random.default_rng(11)
    worst = 0.0
    for _ in range(2000):
        Z = int(rng.integers(1, 27))
        N = int(rng.integers(0, 31))
        A = Z + N
        x = rng.uniform(5.0, 15.0)
        E = 10 ** x * A * MP
        rc, rl, rp = oracle_lib.rates(ot, A, Z, E)
        assert rc == 0
        xc = min(max(math.log10(E / (A * MP)), 6.0), 14.0)
        want = float(I.loss_rate_closed_form(A, Z, xc))
        assert rl == pytest.approx(want, rel=_f32_rate_bound(want, E), abs=0.0)
        worst = max(worst, abs(rl / want - 1.0))
        if A > 1:
            want = float(I.pd_rate_closed_form(A, xc))
            assert rp == pytest.approx(want, rel=_f32_rate_bound(want, E), abs=0.0)
        else:
            assert rp == 0.0
        # the rates are FP32 values, widened exactly
        assert float(np.float32(rl)) == rl and float(np.float32(rp)) == rp
    assert 1e-8 < worst < 4e-5          # FP32 evaluation, not an FP64 one


def test_rates_clamp_to_the_table_ends(oracle_lib):
    """Below and above the tabulated Lorentz factors the end values hold (clamped
    coordinate); E = 0 and E = inf clamp the same way."""
    ot = O.OracleTables(I.synthetic_tables())
    for A, Z in ((56, 26), (4, 2), (1, 1)):
        lo = oracle_lib.rates(ot, A, Z, 10 ** 6 * A * MP)
        hi = oracle_lib.rates(ot, A, Z, 10 ** 14 * A * MP)
        assert oracle_lib.rates(ot, A, Z, 10 ** 3 * A * MP) == lo
        assert oracle_lib.rates(ot, A, Z, 0.0) == lo
        assert oracle_lib.rates(ot, A, Z, 10 ** 17 * A * MP) == hi
        assert oracle_lib.rates(ot, A, Z, math.inf) == hi
        want = float(I.loss_rate_closed_form(A, Z, 6.0))
        assert lo[1] == pytest.approx(want, rel=_f32_rate_bound(want, slope=0.0), abs=0.0)


def test_zero_rate_species_and_range(oracle_lib):
    ot = O.OracleTables(I.synthetic_tables())
    assert oracle_lib.rates(ot, 1, 0, 1e19) == (0, 0.0, 0.0)          # neutron: no loss, no PD
    rc, rl, rp = oracle_lib.rates(ot, 1, 1, 1e19)
    assert rc == 0 and rl > 0 and rp == 0.0                           # proton: loss only
    assert oracle_lib.rates(ot, 60, 27, 1e19)[0] == O.RANGE


def test_continuous_loss_closed_form(oracle_lib):
    """Constant loss rate R: E(s) = E0 exp(-R s); the loss bid keeps steps <= 0.1/R."""
    R = 1.0 / (50 * I.MPC)
    t = I.constant_rate_tables(loss_rate=R)
    dmax = 100 * I.MPC
    st, rc, _ = run(particles([1, 0, 0], 1e19), uniform_grid([0, 0, 0]), I.MPC, dmax, tables=t,
                    hmax=100 * I.MPC)
    assert rc == 0 and st.status[0] == O.DONE
    # the rate the oracle evaluates (FP32, within its bound of R), then the exponential law
    _, Rf, _ = oracle_lib.rates(O.OracleTables(t), 1, 1, 1e19)
    assert Rf == pytest.approx(R, rel=_f32_rate_bound(R, 1e19, slope=0.0), abs=0.0)
    assert st.E[0] == pytest.approx(1e19 * math.exp(-Rf * dmax), rel=1e-13, abs=0.0)
    assert st.n_steps[0] >= 20                                        # 0.1/R = 5 Mpc steps
    assert st.n_int[0] == 0


def test_interaction_counts_are_poisson(oracle_lib):
    """Constant PD rate R over distance D: the count of interactions is Poisson(R D)."""
    R = 1.0 / (20 * I.MPC)
    D = 100 * I.MPC
    t = I.constant_rate_tables(pd_rate=R)
    n = 3000
    rng = np.random.default_rng(3)
    u = rng.standard_normal((n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    st, rc, _ = run(particles(u, 1e20, A=56, Z=26), uniform_grid([0, 0, 0]), I.MPC, D, tables=t,
                    capacity=n * 40, seed=5)
    assert rc == 0
    counts = st.n_int[:n]
    mu = R * D
    kmax = 12
    obs = np.array([np.sum(counts == k) for k in range(kmax)] + [np.sum(counts >= kmax)])
    p = np.array([stats.poisson.pmf(k, mu) for k in range(kmax)] + [stats.poisson.sf(kmax - 1, mu)])
    chi2 = np.sum((obs - n * p) ** 2 / (n * p))
    assert stats.chi2.sf(chi2, len(obs) - 1) > 1e-3
    assert abs(counts.mean() - mu) < 4 * math.sqrt(mu / n)


def test_nucleon_bookkeeping_exact(oracle_lib):
    """Sum of A and of Z over a primary and its secondaries is conserved exactly; with no
    continuous loss the energy is conserved by splits to roundoff."""
    t = I.constant_rate_tables(pd_rate=1.0 / (5 * I.MPC))
    n = 200
    rng = np.random.default_rng(4)
    u = rng.standard_normal((n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    g = I.kolmogorov_grid(16, 0.25 * I.MPC, 2, 8, 1e-13, 2)
    st, rc, stt = run(particles(u, 1e21, A=56, Z=26), g, 0.25 * I.MPC, 200 * I.MPC, tables=t,
                      capacity=n * 56, seed=9)
    assert rc == 0
    s = st.snapshot()
    prim = s["uid"] < 2 ** 32
    parent = np.where(prim, s["uid"], (s["uid"] - 2 ** 32) // 64)
    k = np.where(prim, 0, (s["uid"] - 2 ** 32) % 64)
    assert np.all(s["status"] == O.DONE)
    assert stt["secondaries"] == int(np.sum(~prim)) == int(np.sum(s["n_int"][prim]))
    for pid in range(n):
        sel = parent == pid
        assert int(np.sum(s["A"][sel])) == 56
        assert int(np.sum(s["Z"][sel])) == 26
        assert np.sum(s["E"][sel]) == pytest.approx(1e21, rel=1e-13)
        ks = np.sort(k[sel & ~prim])
        assert np.array_equal(ks, np.arange(1, s["n_int"][pid] + 1))
    sec = ~prim
    assert np.all(s["A"][sec] == 1) and np.all(s["n_int"][sec] == 0)
    assert np.all(s["s"] == 200 * I.MPC)


def test_removed_nucleon_is_proton_with_probability_Z_over_A(oracle_lib):
    t = I.constant_rate_tables(pd_rate=1.0 / I.MPC)
    n = 4000
    st, rc, _ = run(particles(np.tile([1.0, 0, 0], (n, 1)), 1e21, A=56, Z=26), uniform_grid([0, 0, 0]),
                    I.MPC, 0.5 * I.MPC, tables=t, capacity=n * 10, seed=13)
    s = st.snapshot()
    first = (s["uid"] >= 2 ** 32) & ((s["uid"] - 2 ** 32) % 64 == 1)
    frac = np.mean(s["Z"][first] == 1)
    m = int(np.sum(first))
    assert m > 1000
    assert abs(frac - 26 / 56) < 4 * math.sqrt(0.25 / m)


def _c2_like(n=64, seed=2):
    g = I.kolmogorov_grid(16, 0.25 * I.MPC, 2, 8, 1e-13, seed).astype(np.float32)
    p = I.make_particles(n, seed, species=(("H", .4), ("He", .3), ("N", .2), ("Fe", .1)),
                         energy=("power", 1e19, 1e21, 2.0))
    return g, p


def test_budgeted_calls_resume_bit_identically(oracle_lib):
    g, p = _c2_like()
    t = I.synthetic_tables()
    a, rc, _ = run(p, g, 0.25 * I.MPC, 30 * I.MPC, tables=t, capacity=64 * 56)
    assert rc == 0
    f = O.OracleField(g, 0.25 * I.MPC)
    ot = O.OracleTables(t)
    b = O.OracleState(64 * 56)
    O.inject(b, p, 1, ot)
    calls = 0
    while np.any(b.status[:b.n] == O.ACTIVE):
        rc, _ = O.propagate(b, [f], ot, 1e-4, I.KPC, I.MPC, 30 * I.MPC, seed=1, max_steps=37)
        assert rc == 0
        calls += 1
    assert calls > 2
    A, B = _by_uid(a), _by_uid(b)
    for k in A:
        assert np.array_equal(A[k], B[k]), k


def test_thread_count_does_not_change_results(oracle_lib):
    g, p = _c2_like(seed=3)
    t = I.synthetic_tables()
    a, _, _ = run(p, g, 0.25 * I.MPC, 20 * I.MPC, tables=t, capacity=64 * 56, n_threads=1)
    b, _, _ = run(p, g, 0.25 * I.MPC, 20 * I.MPC, tables=t, capacity=64 * 56, n_threads=8)
    A, B = _by_uid(a), _by_uid(b)
    for k in A:
        assert np.array_equal(A[k], B[k]), k


def test_full_secondary_queue_is_resumable(oracle_lib):
    t = I.constant_rate_tables(pd_rate=1.0 / (5 * I.MPC))
    p = particles(np.tile([1.0, 0, 0], (8, 1)), 1e21, A=56, Z=26)
    big, rc, _ = run(p, uniform_grid([0, 0, 1e-13]), I.MPC, 40 * I.MPC, tables=t, capacity=8 * 56)
    assert rc == 0
    f = O.OracleField(uniform_grid([0, 0, 1e-13]), I.MPC)
    ot = O.OracleTables(t)
    small = O.OracleState(9)
    O.inject(small, p, 1, ot)
    rc, _ = O.propagate(small, [f], ot, 1e-4, I.KPC, I.MPC, 40 * I.MPC, seed=1)
    assert rc == O.ERR_QUEUE_FULL
    small.grow(8 * 56)
    rc, _ = O.propagate(small, [f], ot, 1e-4, I.KPC, I.MPC, 40 * I.MPC, seed=1)
    assert rc == 0
    A, B = _by_uid(big), _by_uid(small)
    for k in A:
        assert np.array_equal(A[k], B[k]), k
