"""Differentiation form: the recorded forward and frozen replay are bit-identical to the
oracle; the GPU reverse pass agrees with the oracle's FP64 reverse pass and with central
finite differences (replays on perturbed grids / momenta, steps frozen)."""
import numpy as np
import pytest

import oracle as O
from paper_1410_5323_gb300 import inputs as I

pytestmark = pytest.mark.gpu
C_LIGHT = 299792458.0


def _init(p0, Z):
    """Initial state as the library defines it: E = |p0|, u0 = p0/E, kappa = Z c / E."""
    E = np.sqrt((p0[:, 0] * p0[:, 0] + p0[:, 1] * p0[:, 1]) + p0[:, 2] * p0[:, 2])
    u = p0 / E[:, None]
    return E, u, (Z.astype(np.float64) * C_LIGHT) / E


def _lam(uT, t):
    un = np.linalg.norm(uT, axis=1, keepdims=True)
    uh = uT / un
    gu = 2 * (uh - t)
    return (gu - uh * np.sum(uh * gu, 1, keepdims=True)) / un


def _case(n, grid_n, E0, seed=3):
    g = I.kolmogorov_grid(grid_n, 0.25 * I.MPC, 2, min(32, grid_n // 2), 1e-13, seed).astype(np.float32)
    p = I.make_particles(n, seed + 10, energy=("fixed", E0))
    p0 = p.u * E0
    return g, p.x.copy(), p0, np.ones(n, np.int32)


def test_forward_steps_and_replay_bit_identical_to_oracle(oracle_lib):
    import torch

    import paper_1410_5323_gb300 as crp
    from paper_1410_5323_gb300.adjoint import Adjoint

    g, x0, p0, Z = _case(96, 32, 10 ** 19.5)
    n_steps = 150
    field = crp.Field(torch.from_numpy(g).cuda(), 0.25 * I.MPC)
    adj = Adjoint(field, len(Z), n_steps, 32)
    xT, uT = adj.forward(torch.from_numpy(x0), torch.from_numpy(p0), torch.from_numpy(Z), 1e-4, I.KPC, I.MPC)
    h = adj.steps().cpu().numpy()
    E, u, kap = _init(p0, Z)
    of = O.OracleField(g, 0.25 * I.MPC)
    for i in range(len(Z)):
        y0 = np.concatenate([x0[i], u[i]])
        ho, yT = O.record_steps(of, kap[i], y0, 1e-4, I.KPC, I.MPC, n_steps)
        assert np.array_equal(h[:, i], ho), i
        assert np.array_equal(xT[i].cpu().numpy(), yT[:3]) and np.array_equal(uT[i].cpu().numpy(), yT[3:])
    xr, ur = adj.replay()
    assert torch.equal(xr, xT) and torch.equal(ur, uT)


def test_reverse_pass_matches_oracle_reverse_pass(oracle_lib):
    import torch

    import paper_1410_5323_gb300 as crp
    from paper_1410_5323_gb300.adjoint import Adjoint, perturbed_targets

    g, x0, p0, Z = _case(64, 32, 10 ** 19.5, seed=4)
    n_steps = 200
    field = crp.Field(torch.from_numpy(g).cuda(), 0.25 * I.MPC)
    adj = Adjoint(field, len(Z), n_steps, 64)
    _, uT = adj.forward(torch.from_numpy(x0), torch.from_numpy(p0), torch.from_numpy(Z), 1e-4, I.KPC, I.MPC)
    t = perturbed_targets(uT).cpu().numpy()
    lam = _lam(uT.cpu().numpy(), t)
    gb, pb, xb = adj.backward(torch.from_numpy(lam), g.shape)
    gb, pb, xb = gb.cpu().numpy(), pb.cpu().numpy(), xb.cpu().numpy()
    h = adj.steps().cpu().numpy()
    E, u, kap = _init(p0, Z)
    of = O.OracleField(g, 0.25 * I.MPC)
    go = np.zeros(g.shape)
    for i in range(len(Z)):
        y0 = np.concatenate([x0[i], u[i]])
        yb, kb = O.adjoint(of, kap[i], y0, h[:, i], np.concatenate([np.zeros(3), lam[i]]), go)
        assert np.array_equal(xb[i], yb[:3]), i                # per-particle: same order, same bits
        dot = (u[i, 0] * yb[3] + u[i, 1] * yb[4]) + u[i, 2] * yb[5]
        Eb = -(kb * kap[i]) / E[i]
        pref = (yb[3:] - dot * u[i]) / E[i] + Eb * u[i]
        assert np.array_equal(pb[i], pref), i
    # grid gradient: same terms, summed in another order by the atomics
    assert np.allclose(gb, go, rtol=1e-10, atol=1e-12 * np.abs(go).max())
    assert np.array_equal(gb == 0, go == 0)


def test_reverse_pass_on_a_grid_of_other_sizes(oracle_lib):
    """A non-cubic grid whose sizes are not powers of two (the general index wrap in the
    forward record and the stage records): the same bit-for-bit agreement per particle."""
    import torch

    import paper_1410_5323_gb300 as crp
    from paper_1410_5323_gb300.adjoint import Adjoint, perturbed_targets

    g = (np.random.default_rng(21).standard_normal((12, 10, 14, 3)) * 1e-13).astype(np.float32)
    _, x0, p0, Z = _case(40, 16, 10 ** 19.5, seed=6)
    n_steps = 120
    field = crp.Field(torch.from_numpy(g).cuda(), 0.25 * I.MPC)
    adj = Adjoint(field, len(Z), n_steps, 16)
    _, uT = adj.forward(torch.from_numpy(x0), torch.from_numpy(p0), torch.from_numpy(Z), 1e-4, I.KPC, I.MPC)
    t = perturbed_targets(uT).cpu().numpy()
    lam = _lam(uT.cpu().numpy(), t)
    gb, pb, xb = adj.backward(torch.from_numpy(lam), g.shape)
    gb, xb = gb.cpu().numpy(), xb.cpu().numpy()
    h = adj.steps().cpu().numpy()
    E, u, kap = _init(p0, Z)
    of = O.OracleField(g, 0.25 * I.MPC)
    go = np.zeros(g.shape)
    for i in range(len(Z)):
        y0 = np.concatenate([x0[i], u[i]])
        ho, _ = O.record_steps(of, kap[i], y0, 1e-4, I.KPC, I.MPC, n_steps)
        assert np.array_equal(h[:, i], ho), i
        yb, _ = O.adjoint(of, kap[i], y0, h[:, i], np.concatenate([np.zeros(3), lam[i]]), go)
        assert np.array_equal(xb[i], yb[:3]), i
    assert np.allclose(gb, go, rtol=1e-10, atol=1e-12 * np.abs(go).max())


def test_autograd_function_gives_the_adjoint_gradients(oracle_lib):
    import torch

    from paper_1410_5323_gb300.adjoint import PropagateAdjoint, direction_loss, perturbed_targets

    g, x0, p0, Z = _case(128, 32, 10 ** 19.5, seed=5)
    grid = torch.from_numpy(g).cuda().requires_grad_(True)
    pt = torch.from_numpy(p0).cuda().requires_grad_(True)
    args = (torch.from_numpy(x0).cuda(), torch.from_numpy(Z).cuda(), 0.25 * I.MPC, 120, 32, 1e-4, I.KPC, I.MPC)
    uT = PropagateAdjoint.apply(grid, pt, *args)
    t = perturbed_targets(uT)
    loss = direction_loss(uT, t)
    loss.backward()
    assert grid.grad.shape == grid.shape and grid.grad.dtype == torch.float32
    assert torch.count_nonzero(grid.grad) > 0 and torch.isfinite(grid.grad).all()
    # the same gradients as the adjoint handle driven directly (cast to the input dtypes)
    from paper_1410_5323_gb300.adjoint import Adjoint
    import paper_1410_5323_gb300 as crp

    adj = Adjoint(crp.Field(grid.detach(), 0.25 * I.MPC), len(Z), 120, 32)
    _, uT2 = adj.forward(args[0], pt.detach(), args[1], 1e-4, I.KPC, I.MPC)
    assert torch.equal(uT2, uT.detach())
    u = uT2.clone().requires_grad_(True)
    direction_loss(u, t).backward()
    gb, pb, _ = adj.backward(u.grad, g.shape)
    assert torch.equal(grid.grad, gb.float()) and torch.equal(pt.grad, pb)


@pytest.fixture(scope="module")
def c5():
    import torch

    w = I.workload("adjoint_128cube_4k_protons")
    g = I.kolmogorov_grid(w.grid_n, w.spacing_m, w.lmin_cells, w.lmax_cells, w.brms_t, w.grid_seed).astype(np.float32)
    p = I.make_particles(w.n_particles, w.particle_seed, w.species, w.energy)
    return w, g, p, torch.from_numpy(p.u * 10 ** 19.5), torch.from_numpy(p.x), torch.from_numpy(p.Z)


def test_full_size_reverse_pass_matches_oracle_sampled(c5, oracle_lib):
    """4096 protons at 10^19.5 eV, 128^3 FP32 grid at 1 nG, 2000 frozen steps, checkpoints
    every 64: the whole batch runs on the GPU; 48 sampled particles are rerun by the oracle's
    FP64 reverse pass (steps, x0/p0 gradients bit for bit; their grid gradient to 1e-10)."""
    import torch

    import paper_1410_5323_gb300 as crp
    from paper_1410_5323_gb300.adjoint import Adjoint, perturbed_targets

    w, g, p, p0, x0, Z = c5
    field = crp.Field(torch.from_numpy(g).cuda(), w.spacing_m)
    adj = Adjoint(field, len(p), 2000, 64)
    _, uT = adj.forward(x0, p0, Z, w.tol, w.hmin_m, w.hmax_m)
    t = perturbed_targets(uT)
    lam = _lam(uT.cpu().numpy(), t.cpu().numpy())
    gb_all, pb, xb = adj.backward(torch.from_numpy(lam), g.shape)
    assert torch.isfinite(pb).all() and torch.isfinite(gb_all).all()
    h = adj.steps().cpu().numpy()
    pick = np.sort(np.random.default_rng(0).choice(len(p), 48, replace=False))
    # the sampled particles alone on the GPU, for the grid gradient
    sub = Adjoint(field, len(pick), 2000, 64)
    _, uTs = sub.forward(x0[pick], p0[pick], Z[pick], w.tol, w.hmin_m, w.hmax_m)
    assert torch.equal(uTs, uT[torch.from_numpy(pick).cuda()])
    gbs, _, _ = sub.backward(torch.from_numpy(lam[pick]), g.shape)
    gbs = gbs.cpu().numpy()
    E, u, kap = _init(p0.numpy(), Z.numpy())
    of = O.OracleField(g, w.spacing_m)
    go = np.zeros(g.shape)
    xb, pb = xb.cpu().numpy(), pb.cpu().numpy()
    for i in pick:
        y0 = np.concatenate([x0.numpy()[i], u[i]])
        ho, yT = O.record_steps(of, kap[i], y0, w.tol, w.hmin_m, w.hmax_m, 2000)
        assert np.array_equal(h[:, i], ho)
        yb, kb = O.adjoint(of, kap[i], y0, ho, np.concatenate([np.zeros(3), lam[i]]), go)
        assert np.array_equal(xb[i], yb[:3])
        dot = (u[i, 0] * yb[3] + u[i, 1] * yb[4]) + u[i, 2] * yb[5]
        assert np.array_equal(pb[i], (yb[3:] - dot * u[i]) / E[i] + (-(kb * kap[i]) / E[i]) * u[i])
    assert np.allclose(gbs, go, rtol=1e-10, atol=1e-12 * np.abs(go).max())


def test_adjoint_vs_central_differences_in_the_linear_horizon(c5):
    """Same batch and grid, frozen over the first 200 steps (about 150 Mpc), where the map is
    still linear at representable eps (the trajectories are chaotic: d u_T / d u_0 grows from
    ~1e3 at 200 steps to ~1e24-1e31 at 2000). 32 grid entries with |g| > 1e-3 max|g| and 32
    momentum components. A central difference counts only if its +eps and -eps replays visit
    the same cells as the unperturbed one for every particle (inside a cell the frozen map is
    smooth; across a face the trilinear field is only continuous); two such differences a
    decade apart are Richardson-extrapolated. At least 28 of the 32 must be checkable, and
    those agree with the adjoint to 1e-4."""
    import torch

    import paper_1410_5323_gb300 as crp
    from paper_1410_5323_gb300.adjoint import Adjoint, direction_loss, perturbed_targets

    w, g, p, p0c, x0c, Zc = c5
    p0, x0, Z = p0c.cuda(), x0c.cuda(), Zc.cuda()
    gdev = torch.from_numpy(g).cuda()
    field = crp.Field(gdev, w.spacing_m)
    adj = Adjoint(field, len(p), 200, 64)
    _, uT = adj.forward(x0, p0, Z, w.tol, w.hmin_m, w.hmax_m)
    t = perturbed_targets(uT)
    uT_req = uT.clone().requires_grad_(True)
    direction_loss(uT_req, t).backward()
    gb, pb, _ = adj.backward(uT_req.grad, g.shape)
    gbf = gb.view(-1)
    big = torch.nonzero(gbf.abs() > 1e-3 * gbf.abs().max()).view(-1)
    pick = big[torch.randperm(big.numel(), generator=torch.Generator().manual_seed(0))[:32].to(big.device)]
    g64 = gdev.double()

    _, _, h0 = adj.replay(cells=True)

    def central(run_plus, run_minus, eps):
        """Central difference, or None if a perturbed replay crossed into another cell (the
        trilinear field is only continuous there, so the quotient is no derivative)."""
        _, up, hp = run_plus()
        _, um, hm = run_minus()
        if not (torch.equal(hp, h0) and torch.equal(hm, h0)):
            return None
        return float((direction_loss(up, t) - direction_loss(um, t)) / (2 * eps))

    def grid_run(idx, eps):
        gp = g64.clone().view(-1)
        gp[idx] += eps
        return lambda: adj.replay(crp.Field(gp.view(g64.shape), w.spacing_m), cells=True)

    def derivative(run, scales):
        """Richardson extrapolation of two cell-consistent central differences a decade apart
        (removes the eps^2 term); else the single cell-consistent one; None if none."""
        ds = [(e, central(run(e), run(-e), e)) for e in scales]
        for (e1, d1), (e2, d2) in zip(ds, ds[1:]):
            if d1 is not None and d2 is not None:
                return (100.0 * d2 - d1) / 99.0
        valid = [d for _, d in ds if d is not None]
        return valid[0] if valid else None

    checked, errs = 0, []
    for idx in pick.tolist():
        fd = derivative(lambda e: grid_run(idx, e), [r * 1e-13 for r in (1e-5, 1e-6, 1e-7)])
        if fd is not None:
            checked += 1
            errs.append(abs(fd - float(gbf[idx])) / abs(float(gbf[idx])))
    assert checked >= 28 and max(errs) < 1e-4, ("grid", checked, errs)
    assert int((gbf == 0).sum()) > 0            # entries no stage touched: exactly zero
    pbf = pb.view(-1)

    def p_run(k, eps):
        pp = p0.clone().view(-1)
        pp[k] += eps
        return lambda: adj.replay(p0=pp.view(p0.shape), cells=True)

    checked, errs = 0, []
    for k in torch.randperm(pbf.numel(), generator=torch.Generator().manual_seed(1))[:32].tolist():
        fd = derivative(lambda e: p_run(k, e), [r * 10 ** 19.5 for r in (1e-7, 1e-8, 1e-9)])
        if fd is not None:
            checked += 1
            # relative to the particle's whole gradient vector (a single Cartesian component
            # can be small where the direction and energy parts cancel)
            scale = float(torch.linalg.norm(pb[k // 3]))
            errs.append(abs(fd - float(pbf[k])) / scale)
    assert checked >= 28 and max(errs) < 1e-4, ("momentum", checked, errs)


@pytest.mark.parametrize("n", [1, 7, 13, 31])
def test_team_sweeps_with_partial_teams_match_the_oracle(n, oracle_lib):
    """The forward record and the reverse sweep run three lanes per particle, ten particles
    per warp: batch sizes that leave a warp partly filled give the oracle's steps, arrival
    states and per-particle gradients bit for bit, and its grid gradient to rel 1e-10."""
    import torch

    import paper_1410_5323_gb300 as crp
    from paper_1410_5323_gb300.adjoint import Adjoint

    g, x0, p0, Z = _case(n, 16, 10 ** 19.2, seed=20 + n)
    n_steps = 90
    field = crp.Field(torch.from_numpy(g).cuda(), 0.25 * I.MPC)
    adj = Adjoint(field, n, n_steps, 16)
    xT, uT = adj.forward(torch.from_numpy(x0), torch.from_numpy(p0), torch.from_numpy(Z), 1e-4, I.KPC, I.MPC)
    rng = np.random.default_rng(n)
    lam = rng.standard_normal((n, 3))
    gb, pb, xb = adj.backward(torch.from_numpy(lam), g.shape)
    gb, pb, xb = gb.cpu().numpy(), pb.cpu().numpy(), xb.cpu().numpy()
    h = adj.steps().cpu().numpy()
    E, u, kap = _init(p0, Z)
    of = O.OracleField(g, 0.25 * I.MPC)
    go = np.zeros(g.shape)
    for i in range(n):
        y0 = np.concatenate([x0[i], u[i]])
        ho, yT = O.record_steps(of, kap[i], y0, 1e-4, I.KPC, I.MPC, n_steps)
        assert np.array_equal(h[:, i], ho), i
        assert np.array_equal(xT[i].cpu().numpy(), yT[:3]) and np.array_equal(uT[i].cpu().numpy(), yT[3:])
        yb, kb = O.adjoint(of, kap[i], y0, ho, np.concatenate([np.zeros(3), lam[i]]), go)
        assert np.array_equal(xb[i], yb[:3]), i
        dot = (u[i, 0] * yb[3] + u[i, 1] * yb[4]) + u[i, 2] * yb[5]
        assert np.array_equal(pb[i], (yb[3:] - dot * u[i]) / E[i] + (-(kb * kap[i]) / E[i]) * u[i]), i
    assert np.allclose(gb, go, rtol=1e-10, atol=1e-12 * np.abs(go).max())
    assert np.array_equal(gb == 0, go == 0)
