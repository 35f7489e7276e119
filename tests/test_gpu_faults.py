"""Failure detection without faulting the GPU: the kernels' bounded wait runs out on a flag that
nothing sets and reports a status (the context stays usable), and injected allocation failures
surface as CRP_ERR_OOM with nothing leaked. (Queue overflow, NaN fields and invalid particles
are covered in test_gpu_parity.py.)"""
import numpy as np
import pytest

from paper_1410_5323_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _small_sim(crp, n=64):
    g = I.kolmogorov_grid(8, 0.25 * I.MPC, 2, 4, 1e-13, 1).astype(np.float32)
    sim = crp.Simulation([crp.Field(g, 0.25 * I.MPC)], None, capacity=n)
    sim.inject(I.make_particles(n, 1))
    return sim


def test_bounded_wait_runs_out_and_the_context_stays_usable():
    import paper_1410_5323_gb300 as crp
    from paper_1410_5323_gb300 import api

    assert crp.selftest_wait(1000, preset=-1) == api.ERR_TIMEOUT       # a flag nothing sets
    assert crp.selftest_wait(1000, preset=7) == api.OK                 # a flag already set
    sim = _small_sim(crp)
    sim.propagate(1e-4, I.KPC, I.MPC, 5 * I.MPC)
    assert sim.sync(timeout_s=60.0) == 0
    assert np.all(sim.state()["status"] == crp.STATUS_DONE)


def test_injected_allocation_failures_report_oom_and_leak_nothing():
    import torch

    import paper_1410_5323_gb300 as crp
    from paper_1410_5323_gb300 import api

    g = I.kolmogorov_grid(16, 0.25 * I.MPC, 2, 8, 1e-13, 2).astype(np.float32)
    f = crp.Field(g, 0.25 * I.MPC)           # warm-up allocations outside the measured window
    del f
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for n_fail in (1, 2):
        crp.debug_fail_allocations(n_fail)
        with pytest.raises(crp.CrpError) as e:
            crp.Field(g, 0.25 * I.MPC)        # staging + field: fails on the n-th allocation
        assert e.value.code == api.ERR_OOM
        crp.debug_fail_allocations(0)
    field = crp.Field(g, 0.25 * I.MPC)
    for n_fail in (1, 3, 6, 9):              # state columns, lists, counters, sort scratch
        crp.debug_fail_allocations(n_fail)
        with pytest.raises(crp.CrpError) as e:
            crp.Simulation([field], None, capacity=1000)
        assert e.value.code == api.ERR_OOM
        crp.debug_fail_allocations(0)
    crp.debug_fail_allocations(1)
    with pytest.raises(crp.CrpError) as e:
        crp.Lens(48, np.zeros((1, 49), np.int64), np.zeros(0, np.int32), np.zeros(0, np.float32))
    assert e.value.code == api.ERR_OOM
    crp.debug_fail_allocations(0)
    del field
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free1 - free0) < 16 * 1024 * 1024, (free0, free1)
    sim = _small_sim(crp)                    # the library still works
    sim.propagate(1e-4, I.KPC, I.MPC, 5 * I.MPC)
    assert sim.sync(timeout_s=60.0) == 0


def test_kernel_run_counter_counts_every_launch():
    """crp_kernel_runs counts the library's kernels on the device: injection is two kernels
    (bookkeeping init, slot count); a slot-order propagate call is the prepare kernel, the
    work-list build and two generations of (propagate, swap); the graph loop's kernels are
    counted although the host never launches them one by one."""
    import paper_1410_5323_gb300 as crp
    from paper_1410_5323_gb300 import api

    grid = I.kolmogorov_grid(16, 0.25 * I.MPC, 2, 8, 1e-13, 3).astype(np.float32)
    p = I.make_particles(64, 5)
    sim = crp.Simulation([crp.Field(grid, 0.25 * I.MPC)], None, capacity=len(p))
    nw = crp.kernel_runs()
    sim.inject(p)
    sim.propagate(1e-4, I.KPC, I.MPC, 5 * I.MPC, order=api.ORDER_SLOT)
    sim.sync(60.0)
    assert crp.kernel_runs() - nw == 2 + 6 + 1      # the first FP64-form call also widens the grid
    sim.reset()
    n0 = crp.kernel_runs()
    sim.inject(p)
    assert crp.kernel_runs() - n0 == 2
    n1 = crp.kernel_runs()
    sim.propagate(1e-4, I.KPC, I.MPC, 5 * I.MPC, order=api.ORDER_SLOT)
    sim.sync(60.0)
    assert crp.kernel_runs() - n1 == 6
    sim.reset()
    sim.inject(p)
    n2 = crp.kernel_runs()
    sim.propagate_loop(1e-4, I.KPC, I.MPC, 5 * I.MPC, max_steps=2, order=api.ORDER_SLOT)
    sim.sync(60.0)
    slices = sim.counts()["launches"] // 2
    assert slices > 1
    assert crp.kernel_runs() - n2 >= 6 * slices
