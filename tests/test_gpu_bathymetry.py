"""GPU parity over a varying still-water depth h(x) (Sec. 2.2 sigma map; the bar geometry
of Sec. 6): the six-factor operator, the load vectors with the sloped-bottom arc length,
the slope-free level operators, Schwarz sweeps with per-column factors, the coarse solve,
the V-cycle and full solves, through the C ABI against the oracle.  Tolerances as in
test_gpu_parity."""
from dataclasses import dataclass

import numpy as np
import pytest
import torch

import paper_2411_14977_gb300.pmg as pmg
import workloads as W
from oracle import mg
from oracle.sem import apply_masked, relative_residual, solve_direct
from tests.gpu_helpers import Case, n, t

pytestmark = pytest.mark.gpu


@dataclass
class PeriodicBottom:
    """h(x) = h0 + a sin(2 pi x / L) + b cos(6 pi x / L): a periodic bottom."""
    h0: float
    a: float
    b: float
    L: float

    def __call__(self, x):
        x = np.asarray(x, float)
        return self.h0 + self.a * np.sin(2 * np.pi * x / self.L) + self.b * np.cos(6 * np.pi * x / self.L)

    def slope(self, x):
        x = np.asarray(x, float)
        return (2 * np.pi / self.L) * (self.a * np.cos(2 * np.pi * x / self.L)
                                       - 3 * self.b * np.sin(6 * np.pi * x / self.L))


def periodic_bar(cells_x=8, cells_z=3, order=5):
    L = 0.390625 * cells_x
    s = W.Surface(0.04, 2 * np.pi / L)
    return W.Workload(f"periodic_bottom_{cells_x}x{cells_z}_p{order}", cells_x, cells_z, order, 0.0, L, 1.0, True,
                      W.BASE_SEED + 91, s, "div", velocity=W.Velocity.random(W.BASE_SEED + 92),
                      bathymetry=PeriodicBottom(1.0, 0.25, 0.06, L))


def scaled_bar(cells_x, cells_z, order, rhs="div"):
    """The bar tank on fewer cells (same [0, 36] domain: steeper slopes per cell)."""
    return W.bar(cells_x, cells_z, order, rhs=rhs)


CASES = {
    "bar16x2p6": lambda: scaled_bar(16, 2, 6),
    "bar12x3p5_src": lambda: scaled_bar(12, 3, 5, rhs="source"),
    "bar10x2p8": lambda: scaled_bar(10, 2, 8),
    "periodic8x3p5": lambda: periodic_bar(),
    "bar9x1p4_nz1": lambda: scaled_bar(9, 1, 4),
    "bar1x2p6_nx1": lambda: scaled_bar(1, 2, 6, rhs="source"),
    "bar7x2p2": lambda: scaled_bar(7, 2, 2),
    "bar5x2p10_src": lambda: scaled_bar(5, 2, 10, rhs="source"),
}
_cache = {}


def case(name, **opts):
    key = (name, tuple(sorted(opts.items())))
    if key not in _cache:
        _cache[key] = Case(CASES[name](), **opts)
    return _cache[key]


def scale_of(A, x):
    return np.max(np.abs(A) @ np.abs(x))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("df64", [0, 1])
def test_apply_over_varying_depth(name, df64):
    c = case(name, df64_outer=df64)
    A = c.m.assemble(c.eta)
    x = np.random.default_rng(21).standard_normal(c.m.N)
    dm = c.m.dirichlet_mask()
    ref = apply_masked(A, x, dm)
    s = scale_of(A, np.where(dm, 0, x))
    assert np.max(np.abs(n(c.S.apply(t(x))) - ref)) <= 1e-12 * s
    assert np.max(np.abs(n(c.S.apply_f32(t(x, torch.float32))) - ref)) <= 2e-5 * s


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_over_varying_depth(name):
    c = case(name)
    ref = c.rhs_oracle()
    b = n(c.rhs_gpu())
    assert np.max(np.abs(b - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("flat", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_level_operators_over_varying_depth(name, flat):
    """Slope-free level operators with per-element x-stiffness (slab or node-parallel)."""
    c = case(name, flat_kernel=flat)
    H = c.hierarchy()
    rng = np.random.default_rng(22)
    for l, lev in enumerate(H.levels):
        x = rng.standard_normal(lev.mesh.N)
        x[lev.dmask] = 0.0
        ref = lev.A @ x[lev.free]
        s = np.max(np.abs(lev.A) @ np.abs(x[lev.free]))
        for dt, tol in ((torch.float64, 1e-12), (torch.float32, 2e-5)):
            y = n(c.S.level_apply(l, t(x, dt)))
            assert np.max(np.abs(y[lev.free] - ref)) <= tol * s, (l, dt)


@pytest.mark.parametrize("name", list(CASES))
def test_smoother_over_varying_depth(name):
    """Schwarz sweeps with one x-factorisation per element column: the fast-diagonalisation
    inverse equals the oracle's dense Cholesky of each subdomain block."""
    c = case(name)
    H = c.hierarchy()
    rng = np.random.default_rng(23)
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
def test_coarse_solve_and_vcycle_over_varying_depth(name):
    c = case(name)
    H = c.hierarchy()
    rng = np.random.default_rng(24)
    C = H.levels[-1]
    b = rng.standard_normal(C.mesh.N)
    b[C.dmask] = 0.0
    ref = np.zeros(C.mesh.N)
    ref[C.free] = H.coarse_lu.solve(b[C.free])
    assert np.max(np.abs(n(c.S.coarse_solve(t(b))) - ref)) <= 1e-11 * np.max(np.abs(ref))
    F = H.levels[0]
    r = rng.standard_normal(F.mesh.N)
    r[F.dmask] = 0.0
    zref = np.zeros(F.mesh.N)
    zref[F.free] = H.vcycle(r[F.free])
    assert np.max(np.abs(n(c.S.vcycle(t(r))) - zref)) <= 1e-10 * np.max(np.abs(zref))
    assert np.max(np.abs(n(c.S.vcycle(t(r, torch.float32))) - zref)) <= 1e-4 * np.max(np.abs(zref))


VARIANTS = [dict(), dict(outer=pmg.PMG_FCG), dict(precision=pmg.PMG_MIXED_FP32),
            dict(precision=pmg.PMG_MIXED_FP32, outer=pmg.PMG_IR), dict(outer=pmg.PMG_GMRES),
            dict(precision=pmg.PMG_MIXED_FP32, flat_kernel=1), dict(precision=pmg.PMG_MIXED_FP32, outer=pmg.PMG_GMRES)]


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("variant", VARIANTS)
def test_solve_over_varying_depth(name, variant):
    c = Case(CASES[name](), tol=1e-12, **variant)
    bo = c.rhs_oracle()
    A = c.m.assemble(c.eta)
    dm = c.m.dirichlet_mask()
    pref = solve_direct(A, bo, c.F["pD"], dm)
    p, info = c.S.solve(c.rhs_gpu(), t(c.F["pD"]))
    p = n(p)
    err = np.linalg.norm(p - pref) / np.linalg.norm(pref)
    assert err <= 1e-10, (err, info)
    assert info["rel_residual"] <= 1e-12
    assert relative_residual(A, bo, p, dm) <= 2e-12
    np.testing.assert_array_equal(p[dm], c.F["pD"][dm])
    if not variant:
        # FP64 PCG: the oracle's PCG with the same (slope-free, per-column depth) V-cycle
        _, its, _, _ = mg.solve(c.m, c.eta, bo, c.F["pD"], tol=1e-12, overlap=1, nu=2, omega=0.8)
        assert abs(info["iterations"] - its) <= 1, (info["iterations"], its)


def test_constant_depth_through_bathymetry_matches_constant_mesh():
    """A constant depth given per column reproduces the constant-depth handle: operator
    to rounding, the same V-cycle (per-column tables equal the class tables), the same
    iteration count."""
    w = W.tank(12, 3, 6)
    a = Case(w)
    b = Case(w)
    b.S.set_bathymetry(t(np.full(b.m.NX, w.h)))
    b.S.set_geometry(t(b.eta))
    x = np.random.default_rng(25).standard_normal(a.m.N)
    ya, yb = n(a.S.apply(t(x))), n(b.S.apply(t(x)))
    assert np.max(np.abs(ya - yb)) <= 1e-13 * np.max(np.abs(ya))
    r = x.copy()
    r[a.m.dirichlet_mask()] = 0.0
    za, zb = n(a.S.vcycle(t(r))), n(b.S.vcycle(t(r)))
    assert np.max(np.abs(za - zb)) <= 1e-11 * np.max(np.abs(za))
    pa, ia = a.S.solve(a.rhs_gpu(), t(a.F["pD"]))
    pb, ib = b.S.solve(b.rhs_gpu(), t(b.F["pD"]))
    assert abs(ia["iterations"] - ib["iterations"]) <= 1
    assert np.max(np.abs(n(pa) - n(pb))) <= 1e-9 * np.max(np.abs(n(pa)))


def test_autotune_over_varying_depth():
    c = Case(scaled_bar(24, 2, 6), tol=1e-11, precision=pmg.PMG_MIXED_FP32)
    c.S.autotune()
    bo = c.rhs_oracle()
    A = c.m.assemble(c.eta)
    dm = c.m.dirichlet_mask()
    pref = solve_direct(A, bo, c.F["pD"], dm)
    p, info = c.S.solve(c.rhs_gpu(), t(c.F["pD"]))
    assert np.linalg.norm(n(p) - pref) / np.linalg.norm(pref) <= 1e-9


def test_varying_depth_rejections():
    w = scaled_bar(6, 2, 4)
    c = Case(w)
    with pytest.raises(pmg.PmgError):
        c.S.set_geometry_mixed(t(c.eta), t(c.eta))
    S = pmg.Solver(**w.mesh_kwargs())
    xc, _ = S.node_coords()
    bad = w.depth(xc)
    bad[3] = -0.1
    with pytest.raises(pmg.PmgError):
        S.set_bathymetry(t(bad))
    S.close()
    S = pmg.Solver(**w.mesh_kwargs(), precision=pmg.PMG_MIXED_BF16, outer=pmg.PMG_IR)
    with pytest.raises(pmg.PmgError):
        S.set_bathymetry(t(w.depth(xc)))
    S.close()
