"""GPU parity of the dense additive-Schwarz smoother (PMG_ASM_DENSE: subdomain blocks of
the assembled level matrix inverted on the device, Sec. 5.3) against the oracle, whose
smoother is the same definition by dense Cholesky: sweeps, V-cycle, solves with the
oracle's iteration counts, and the same results as fast diagonalisation."""
import numpy as np
import pytest
import torch

import paper_2411_14977_gb300.pmg as pmg
import workloads as W
from oracle import mg
from oracle.sem import solve_direct
from tests.gpu_helpers import Case, n, t
from tests.test_gpu_parity import periodic_tank

pytestmark = pytest.mark.gpu

CASES = {
    "tank12x3p6": lambda: W.tank(12, 3, 6),
    "cfg1": lambda: W.config1(),
    "periodic8x3p5": lambda: periodic_tank(),
    "tank6x2p8": lambda: W.tank(6, 2, 8),
    "tank7x3p2": lambda: W.tank(7, 3, 2),
    "bar12x2p6": lambda: W.bar(12, 2, 6),
    "p4z8": lambda: W.paper_scaling(10, 4, order_z=8),
    "tank1x2p5_nx1": lambda: W.tank(1, 2, 5),
    "tank5x1p4_nz1": lambda: W.tank(5, 1, 4),
}
_cache = {}


def case(name, **opts):
    key = (name, tuple(sorted(opts.items())))
    if key not in _cache:
        _cache[key] = Case(CASES[name](), smoother=pmg.PMG_ASM_DENSE, **opts)
    return _cache[key]


@pytest.mark.parametrize("name", list(CASES))
def test_dense_smoother_matches_oracle(name):
    c = case(name)
    H = c.hierarchy()
    rng = np.random.default_rng(51)
    for l, lev in enumerate(H.levels[:-1]):
        N = lev.mesh.N
        b = rng.standard_normal(N)
        b[lev.dmask] = 0.0
        x0 = rng.standard_normal(N)
        x0[lev.dmask] = 0.0
        for post in (False, True):
            ref = np.zeros(N)
            ref[lev.free] = H.smooth(l, b[lev.free], x0[lev.free], post)
            sc = max(1.0, np.max(np.abs(ref)))
            for dt, tol in ((torch.float64, 1e-11), (torch.float32, 1e-4)):
                x = c.S.level_smooth(l, t(b, dt), t(x0, dt), post)
                assert np.max(np.abs(n(x) - ref)) <= tol * sc, (l, post, dt)


@pytest.mark.parametrize("name", list(CASES))
def test_dense_vcycle_matches_oracle(name):
    c = case(name)
    H = c.hierarchy()
    F = H.levels[0]
    r = np.random.default_rng(52).standard_normal(F.mesh.N)
    r[F.dmask] = 0.0
    zref = np.zeros(F.mesh.N)
    zref[F.free] = H.vcycle(r[F.free])
    assert np.max(np.abs(n(c.S.vcycle(t(r))) - zref)) <= 1e-10 * np.max(np.abs(zref))
    assert np.max(np.abs(n(c.S.vcycle(t(r, torch.float32))) - zref)) <= 1e-4 * np.max(np.abs(zref))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("variant", [dict(), dict(precision=pmg.PMG_MIXED_FP32), dict(outer=pmg.PMG_GMRES)])
def test_dense_solve_matches_direct_and_oracle_iterations(name, variant):
    c = Case(CASES[name](), tol=1e-12, smoother=pmg.PMG_ASM_DENSE, **variant)
    bo = c.rhs_oracle()
    A = c.m.assemble(c.eta)
    dm = c.m.dirichlet_mask()
    pref = solve_direct(A, bo, c.F["pD"], dm)
    p, info = c.S.solve(c.rhs_gpu(), t(c.F["pD"]))
    assert np.linalg.norm(n(p) - pref) / np.linalg.norm(pref) <= 1e-10
    if not variant:
        _, its, _, _ = mg.solve(c.m, c.eta, bo, c.F["pD"], tol=1e-12, overlap=1, nu=2, omega=0.8)
        assert abs(info["iterations"] - its) <= 1, (info["iterations"], its)
        # the same V-cycle as fast diagonalisation (both invert the same blocks)
        f = Case(CASES[name](), tol=1e-12)
        _, info_f = f.S.solve(f.rhs_gpu(), t(f.F["pD"]))
        assert abs(info["iterations"] - info_f["iterations"]) <= 1


def test_dense_order_ten_blocks_fit_and_solve():
    """Order 10 with overlap 1: 169 x 169 FP64 blocks (228,488 bytes) fit one CTA's shared
    memory; the solve matches the direct solution."""
    c = Case(W.tank(4, 2, 10), tol=1e-12, smoother=pmg.PMG_ASM_DENSE)
    bo = c.rhs_oracle()
    A = c.m.assemble(c.eta)
    dm = c.m.dirichlet_mask()
    pref = solve_direct(A, bo, c.F["pD"], dm)
    p, info = c.S.solve(c.rhs_gpu(), t(c.F["pD"]))
    assert np.linalg.norm(n(p) - pref) / np.linalg.norm(pref) <= 1e-10


ACTUAL_CASES = ["tank12x3p6", "periodic8x3p5", "tank6x2p8", "tank7x3p2", "cfg1"]


@pytest.mark.parametrize("name", ACTUAL_CASES)
def test_actual_geometry_levels_match_oracle(name):
    """PMG_ACTUAL: every level but the order-1 one on the current surface (Sec. 5: the
    preconditioner re-discretised instead of frozen), dense Schwarz inverses rebuilt at each
    pmg_set_geometry; the oracle's hierarchy with geometry='actual', coarsest level flat."""
    c = Case(CASES[name](), tol=1e-12, smoother=pmg.PMG_ASM_DENSE, precond_geom=pmg.PMG_ACTUAL)
    H = mg.Hierarchy(c.m, c.eta, overlap=1, nu=2, omega=0.8, geometry='actual', coarse_geometry='flat')
    rng = np.random.default_rng(53)
    for l, lev in enumerate(H.levels):
        x = rng.standard_normal(lev.mesh.N)
        x[lev.dmask] = 0.0
        ref = lev.A @ x[lev.free]
        s = np.max(np.abs(lev.A) @ np.abs(x[lev.free]))
        for dt, tol in ((torch.float64, 1e-12), (torch.float32, 2e-5)):
            y = n(c.S.level_apply(l, t(x, dt)))
            assert np.max(np.abs(y[lev.free] - ref)) <= tol * s, (l, dt)
    F0 = H.levels[0]
    r = rng.standard_normal(F0.mesh.N)
    r[F0.dmask] = 0.0
    zref = np.zeros(F0.mesh.N)
    zref[F0.free] = H.vcycle(r[F0.free])
    assert np.max(np.abs(n(c.S.vcycle(t(r))) - zref)) <= 1e-10 * np.max(np.abs(zref))
    bo = c.rhs_oracle()
    p, info = c.S.solve(c.rhs_gpu(), t(c.F["pD"]))
    pref = solve_direct(c.m.assemble(c.eta), bo, c.F["pD"], c.m.dirichlet_mask())
    assert np.linalg.norm(n(p) - pref) / np.linalg.norm(pref) <= 1e-10
    _, its, _, _ = mg.solve(c.m, c.eta, bo, c.F["pD"], hier=H, tol=1e-12)
    assert abs(info["iterations"] - its) <= 1, (info["iterations"], its)
    # a new surface: the levels follow it
    eta2 = 1.5 * c.eta[::-1].copy() if not c.w.periodic else np.roll(c.eta, 3)
    c.S.set_geometry(t(eta2))
    H2 = mg.Hierarchy(c.m, eta2, overlap=1, nu=2, omega=0.8, geometry='actual', coarse_geometry='flat')
    zref2 = np.zeros(F0.mesh.N)
    zref2[F0.free] = H2.vcycle(r[F0.free])
    assert np.max(np.abs(n(c.S.vcycle(t(r))) - zref2)) <= 1e-10 * np.max(np.abs(zref2))


def test_actual_geometry_needs_dense_blocks():
    with pytest.raises(pmg.PmgError):
        pmg.Solver(6, 2, 4, precond_geom=pmg.PMG_ACTUAL)
    S = pmg.Solver(6, 2, 4, precond_geom=pmg.PMG_ACTUAL, smoother=pmg.PMG_ASM_DENSE)
    with pytest.raises(pmg.PmgError):
        S.set_bathymetry(torch.ones(S.NX, dtype=torch.float64, device="cuda"))
    S.close()
