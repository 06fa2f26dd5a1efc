"""Parity of the bulk-staged FP32 level operator (slab CTAs whose x slab and b run are staged
by 16-byte-aligned TMA bulk copies, the ragged head and tail by plain loads;
pmg_opts.flat_kernel = 3 or 1000 + threads) against the oracle's assembled level matrices
(Sec. 5: the flat Kronecker-sum level), on walled and periodic meshes of every order down to
1 (the periodic slab wraps at both ends of the tank; 1-column and 1-row tanks; odd and even
column heights, so runs start at every offset modulo four floats); its residual form inside
the Schwarz smoothing against the slab kernel's; solves through it; and its bounded wait."""
import numpy as np
import pytest
import torch

import paper_2411_14977_gb300.pmg as pmg
import workloads as W
from oracle.sem import solve_direct

from gpu_helpers import Case, n, t

pytestmark = pytest.mark.gpu

CODES = [3, 1064, 1512]


def periodic_tank(cells_x, cells_z, order):
    L = 0.390625 * cells_x
    s = W.Surface(0.04, 2 * np.pi / L)
    return W.Workload(f"periodic_{cells_x}x{cells_z}_p{order}", cells_x, cells_z, order, 0.0, L, 1.0, True,
                      W.BASE_SEED + 93, s, "div", velocity=W.Velocity.random(W.BASE_SEED + 94))


MESHES = {
    "tank37x11p6": lambda: W.tank(37, 11, 6),
    "tank20x9p8": lambda: W.tank(20, 9, 8),
    "tank9x3p7": lambda: W.tank(9, 3, 7),
    "tank6x4p10": lambda: W.tank(6, 4, 10),
    "periodic32x9p4": lambda: periodic_tank(32, 9, 4),
    "periodic4x5p5": lambda: periodic_tank(4, 5, 5),
    "tank1x1p2": lambda: W.tank(1, 1, 2),
    "tank3x1p3": lambda: W.tank(3, 1, 3),
}
_hier = {}


def hierarchy(name, c):
    if name not in _hier:
        _hier[name] = c.hierarchy()
    return _hier[name]


@pytest.mark.parametrize("code", CODES)
@pytest.mark.parametrize("name", list(MESHES))
def test_bulk_level_operator_matches_oracle(name, code):
    """y = A_l x on every level in FP32: free rows against the oracle's A_l (the surface row
    of x is read as zero), surface rows pass x through."""
    c = Case(MESHES[name](), precision=pmg.PMG_MIXED_FP32, flat_kernel=code)
    for l in range(c.S.nlevels):
        assert c.S.level_kernels(l)["flat32"] == (1256 if code == 3 else code)
    H = hierarchy(name, c)
    rng = np.random.default_rng(6)
    for l, lev in enumerate(H.levels):
        x = rng.standard_normal(lev.mesh.N)
        x32 = x.astype(np.float32).astype(np.float64)
        y = n(c.S.level_apply(l, t(x32, torch.float32)))
        xf = x32.copy()
        xf[lev.dmask] = 0.0
        ref = lev.A @ xf[lev.free]
        s = np.max(np.abs(lev.A) @ np.abs(xf[lev.free]))
        assert np.max(np.abs(y[lev.free] - ref)) <= 2e-5 * s, (l, lev.mesh.P)
        np.testing.assert_array_equal(y[lev.dmask], x32[lev.dmask])


@pytest.mark.parametrize("name", ["tank37x11p6", "periodic32x9p4", "periodic4x5p5", "tank1x1p2"])
def test_bulk_residual_in_smoothing_matches_slab(name):
    """nu sweeps from a nonzero start (each after a level residual b - A_l x) agree with the
    same sweeps after the slab kernel's residual to FP32 rounding."""
    w = MESHES[name]()
    out = {}
    for fk in (0, 3):
        c = Case(w, precision=pmg.PMG_MIXED_FP32, flat_kernel=fk)
        rng = np.random.default_rng(8)
        res = []
        for l in range(c.S.nlevels - 1):
            NX, NZ = c.S.level_info(l)[1:]
            b = rng.standard_normal(NX * NZ).astype(np.float32)
            x = rng.standard_normal(NX * NZ).astype(np.float32)
            b.reshape(NX, NZ)[:, -1] = 0.0
            x.reshape(NX, NZ)[:, -1] = 0.0
            xd = t(x, torch.float32)
            c.S.level_smooth(l, t(b, torch.float32), xd, post=bool(l % 2))
            res.append(n(xd))
        out[fk] = res
    for a, b in zip(out[0], out[3]):
        assert np.max(np.abs(a - b)) <= 2e-5 * np.max(np.abs(a))


@pytest.mark.parametrize("name", ["tank37x11p6", "periodic32x9p4", "tank6x4p10"])
def test_solve_through_bulk_levels(name):
    w = MESHES[name]()
    runs = {}
    for fk in (0, 3):
        c = Case(w, tol=1e-10, precision=pmg.PMG_MIXED_FP32, flat_kernel=fk)
        p, info = c.S.solve(c.rhs_gpu(), t(c.F["pD"]))
        assert info["status"] == 0 and info["rel_residual"] <= 1e-10, (fk, info)
        runs[fk] = (n(p), info["iterations"])
    pref = solve_direct(c.m.assemble(c.eta), c.rhs_oracle(), c.F["pD"], c.m.dirichlet_mask())
    assert abs(runs[3][1] - runs[0][1]) <= 1, runs
    for fk, (p, _) in runs.items():
        assert np.max(np.abs(p - pref)) <= 1e-7 * np.max(np.abs(pref)), fk


def test_bulk_wait_limit_reports_timeout_and_recovers():
    """A wait limit of zero cycles: every CTA of the bulk-staged residual gives up on its
    mbarrier at once, raises the flag, waits for its copies and leaves y unwritten; the
    solve reports PMG_ERR_TIMEOUT and solves again with the limit restored."""
    c = Case(MESHES["tank37x11p6"](), precision=pmg.PMG_MIXED_FP32, tol=1e-10, max_iter=30, flat_kernel=3,
             sweep_kernel=0)
    b, pD = c.rhs_gpu(), t(c.F["pD"])
    c.S.set_wait_limit(0)
    with pytest.raises(pmg.PmgError) as e:
        c.S.solve(b, pD)
    assert e.value.status == pmg.PMG_ERR_TIMEOUT
    c.S.set_wait_limit(-1)
    p, info = c.S.solve(b, pD)
    assert info["status"] == pmg.PMG_OK and info["rel_residual"] <= 1e-10
