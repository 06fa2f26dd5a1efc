"""Fused coarse V-cycle: the FP32 V-cycle's levels of order <= 4 and the order-1 coarse
solve (Sec. 5) in one cooperative launch, its steps separated by grid barriers with
bounded waits.

* It computes the V-cycle of the launch-per-step path (the steps are recorded from that
  path and run by the same device bodies), element by element against the path itself
  and against the oracle's V-cycle, on walled, periodic, one-column, one-row and
  bench-shaped tanks of orders 2..10.
* A grid barrier whose wait runs out reports PMG_ERR_TIMEOUT (wait limit 0 cycles: every
  CTA but the last to arrive gives up at once); nothing faults, and the handle solves again
  once the limit is restored.
* With it, one outer iteration of the mixed solve launches at most 20 kernels.
* It is opt-in (pmg_opts.fuse_coarse = 1, or pmg_autotune where the whole FP32 V-cycle
  measures faster with it): on a GB300 its grid barriers cost more than the kernel
  boundaries they replace.
"""
import numpy as np
import pytest
import torch

import paper_2411_14977_gb300.pmg as pmg
import workloads as W
from oracle.sem import solve_direct
from tests.gpu_helpers import Case, n, t
from tests.test_gpu_parity import periodic_tank

pytestmark = pytest.mark.gpu

CASES = {
    "tank12x3p6": lambda: W.tank(12, 3, 6),
    "periodic8x3p5": lambda: periodic_tank(),
    "tank6x2p8": lambda: W.tank(6, 2, 8),
    "tank5x1p4_nz1": lambda: W.tank(5, 1, 4),
    "tank1x2p5_nx1": lambda: W.tank(1, 2, 5),
    "tank4x2p10": lambda: W.tank(4, 2, 10),
    "tank7x3p2": lambda: W.tank(7, 3, 2),
    "slice32x32p6": lambda: W.tank(32, 32, 6),
}


def first_fused_level(orders):
    """Index of the first level the fused kernel covers: the levels of order <= 4 below the
    finest, down to the coarse level (which is always covered)."""
    l0 = len(orders) - 1
    while l0 - 1 >= 1 and orders[l0 - 1] <= 4:
        l0 -= 1
    return l0


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("flat_kernel", [-1, 1])
def test_fused_vcycle_matches_stepwise_and_oracle(name, flat_kernel):
    c = Case(CASES[name](), precision=pmg.PMG_MIXED_FP32, flat_kernel=flat_kernel, fuse_coarse=1)
    orders = [c.S.level_info(l)[0] for l in range(c.S.nlevels)]
    info = c.S.fused_vcycle_info()
    assert info["first_level"] == first_fused_level(orders)
    assert info["on"] == 1
    H = c.hierarchy()
    F = H.levels[0]
    rng = np.random.default_rng(11)
    r = rng.standard_normal(F.mesh.N)
    r[F.dmask] = 0.0
    zref = np.zeros(F.mesh.N)
    zref[F.free] = H.vcycle(r[F.free])
    z_on = n(c.S.vcycle(t(r, torch.float32)))
    c.S.set_fused_vcycle(0)
    z_off = n(c.S.vcycle(t(r, torch.float32)))
    c.S.set_fused_vcycle(1)
    z_again = n(c.S.vcycle(t(r, torch.float32)))
    # deterministic: the same launch twice gives the same bits
    assert np.array_equal(z_on, z_again)
    scale = np.max(np.abs(zref))
    # the same steps in FP32; the level residual may be the slab or the node-parallel
    # kernel on the launch-per-step path (the fused one is node-parallel): rounding order
    assert np.max(np.abs(z_on - z_off)) <= 2e-6 * scale
    assert np.max(np.abs(z_on - zref)) <= 1e-4 * scale


@pytest.mark.parametrize("name", ["tank12x3p6", "slice32x32p6", "periodic8x3p5"])
def test_fused_solve_matches_direct(name):
    # FP64-pipe outer operator: 1e-11 is below the double-float operator's residual floor
    # on the 32-row slice
    c = Case(CASES[name](), precision=pmg.PMG_MIXED_FP32, tol=1e-11, fuse_coarse=1, df64_outer=0)
    assert c.S.fused_vcycle_info()["on"] == 1
    b, pD = c.rhs_gpu(), t(c.F["pD"])
    p, info = c.S.solve(b, pD)
    assert info["status"] == pmg.PMG_OK and info["rel_residual"] <= 1e-11
    pref = solve_direct(c.m.assemble(c.eta), c.rhs_oracle(), c.F["pD"], c.m.dirichlet_mask())
    assert np.linalg.norm(n(p) - pref) <= 1e-9 * np.linalg.norm(pref)


def test_fused_off_by_option_and_default():
    c = Case(W.tank(12, 3, 6), precision=pmg.PMG_MIXED_FP32, fuse_coarse=0)
    info = c.S.fused_vcycle_info()
    assert info["first_level"] == -1 and info["on"] == 0
    with pytest.raises(pmg.PmgError):
        c.S.set_fused_vcycle(1)
    # default: built, off until the autotuner measures it faster (a mesh no other test tunes:
    # the decision is remembered per mesh shape for the process)
    c = Case(W.tank(13, 3, 6), precision=pmg.PMG_MIXED_FP32)
    info = c.S.fused_vcycle_info()
    assert info["first_level"] == 1 and info["on"] == 0
    c.S.autotune()
    info = c.S.fused_vcycle_info()
    assert info["us_off"] > 0 and info["us_on"] > 0
    assert info["on"] == int(info["us_on"] < 0.97 * info["us_off"])


def test_fused_grid_barrier_timeout_reports_and_recovers():
    # slab sweeps: the only bounded waits of the solve are the fused kernel's grid barriers
    c = Case(W.tank(12, 3, 6), precision=pmg.PMG_MIXED_FP32, tol=1e-11, max_iter=40, sweep_kernel=0,
             fuse_coarse=1)
    assert c.S.fused_vcycle_info()["on"] == 1
    b, pD = c.rhs_gpu(), t(c.F["pD"])
    c.S.set_wait_limit(0)
    with pytest.raises(pmg.PmgError) as e:
        c.S.solve(b, pD)
    assert e.value.status == pmg.PMG_ERR_TIMEOUT
    c.S.set_wait_limit(-1)
    p, info = c.S.solve(b, pD)
    assert info["status"] == pmg.PMG_OK and info["rel_residual"] <= 1e-11
    pref = solve_direct(c.m.assemble(c.eta), c.rhs_oracle(), c.F["pD"], c.m.dirichlet_mask())
    assert np.linalg.norm(n(p) - pref) <= 1e-9 * np.linalg.norm(pref)


def test_launches_per_outer_iteration():
    c = Case(W.tank(32, 32, 6), precision=pmg.PMG_MIXED_FP32, tol=1e-10, fuse_coarse=1)
    b, pD = c.rhs_gpu(), t(c.F["pD"])
    c.S.solve(b, pD)
    c.S.profile_reset(timing=False)
    _, info = c.S.solve(b, pD)
    launches = sum(v[0] for v in c.S.profile_read().values())
    it = info["iterations"]
    assert it >= 5
    # setup of the solve (lifting, first residual, initial direction, final residual) and
    # at most 20 launches per iteration
    assert launches <= 20 * it + 20, (launches, it)
    c.S.set_fused_vcycle(0)
    c.S.profile_reset(timing=False)
    _, info2 = c.S.solve(b, pD)
    launches2 = sum(v[0] for v in c.S.profile_read().values())
    assert info2["iterations"] == it
    assert launches2 > launches
