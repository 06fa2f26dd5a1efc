"""Parity of the tiled FP32 level operator (one thread per element, CTAs of EXT element
columns x ZT element rows, pmg_opts.flat_kernel = 2 or a shape code 10000 + 100 EXT + ZT)
against the oracle's assembled level matrices (Sec. 5: the flat Kronecker-sum level), on
meshes that span several tiles with ragged last tiles in both directions, walled and
periodic (power-of-two column counts; 16 columns leave a ragged 32-column tile), and
every level order down to 1; then solves through it."""
import numpy as np
import pytest
import torch

import paper_2411_14977_gb300.pmg as pmg
import workloads as W
from oracle.sem import solve_direct

from gpu_helpers import Case, n, t

pytestmark = pytest.mark.gpu

CODES = [2, 10804, 10808, 11604, 11608, 13204, 13208]


def periodic_tank(cells_x, cells_z, order):
    L = 0.390625 * cells_x
    s = W.Surface(0.04, 2 * np.pi / L)
    return W.Workload(f"periodic_{cells_x}x{cells_z}_p{order}", cells_x, cells_z, order, 0.0, L, 1.0, True,
                      W.BASE_SEED + 91, s, "div", velocity=W.Velocity.random(W.BASE_SEED + 92))


MESHES = {
    "tank37x11p6": lambda: W.tank(37, 11, 6),
    "tank70x9p8": lambda: W.tank(70, 9, 8),
    "tank9x3p7": lambda: W.tank(9, 3, 7),
    "periodic32x9p4": lambda: periodic_tank(32, 9, 4),
    "periodic16x5p5": lambda: periodic_tank(16, 5, 5),
    "tank1x1p2": lambda: W.tank(1, 1, 2),
}
_hier = {}


def hierarchy(name, c):
    if name not in _hier:
        _hier[name] = c.hierarchy()
    return _hier[name]


@pytest.mark.parametrize("code", CODES)
@pytest.mark.parametrize("name", list(MESHES))
def test_tiled_level_operator_matches_oracle(name, code):
    """y = A_l x on every level in FP32: free rows against the oracle's A_l (the surface row
    of x is read as zero), surface rows pass x through."""
    c = Case(MESHES[name](), precision=pmg.PMG_MIXED_FP32, flat_kernel=code)
    H = hierarchy(name, c)
    rng = np.random.default_rng(5)
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


@pytest.mark.parametrize("code", [2, 13208, 10804])
@pytest.mark.parametrize("name", ["tank37x11p6", "periodic32x9p4"])
def test_solve_through_tiled_levels(name, code):
    """The mixed-precision solve to 1e-10 with the tiled level residual (b - A_l x) in its
    V-cycle takes the iterations of the same solve with slab-CTA levels (within one) and
    reaches the direct FP64 solution."""
    w = MESHES[name]()
    runs = {}
    for fk in (0, code):
        c = Case(w, tol=1e-10, precision=pmg.PMG_MIXED_FP32, flat_kernel=fk)
        p, info = c.S.solve(c.rhs_gpu(), t(c.F["pD"]))
        assert info["status"] == 0 and info["rel_residual"] <= 1e-10, (fk, info)
        runs[fk] = (n(p), info["iterations"])
    bo = c.rhs_oracle()
    pref = solve_direct(c.m.assemble(c.eta), bo, c.F["pD"], c.m.dirichlet_mask())
    assert abs(runs[code][1] - runs[0][1]) <= 1, runs
    for fk, (p, _) in runs.items():
        assert np.max(np.abs(p - pref)) <= 1e-7 * np.max(np.abs(pref)), fk


def test_autotuned_levels_match_oracle():
    """The autotuner's free choice (slab, node-parallel or tiled per level) keeps parity."""
    c = Case(MESHES["tank37x11p6"](), precision=pmg.PMG_MIXED_FP32)
    c.S.autotune()
    H = hierarchy("tank37x11p6", c)
    rng = np.random.default_rng(6)
    for l, lev in enumerate(H.levels):
        x = rng.standard_normal(lev.mesh.N)
        x[lev.dmask] = 0.0
        y = n(c.S.level_apply(l, t(x, torch.float32)))
        ref = lev.A @ x[lev.free]
        s = np.max(np.abs(lev.A) @ np.abs(x[lev.free]))
        assert np.max(np.abs(y[lev.free] - ref)) <= 2e-5 * s, l
