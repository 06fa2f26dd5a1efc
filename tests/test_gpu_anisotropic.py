"""GPU parity with different polynomial orders along x and sigma (Sec. 5.1 semi-coarsening;
the scaling study of Sec. 6.3 runs P_z = 8 with P_x = 2..10): operator, load vectors,
level operators, transfers, Schwarz sweeps, coarse solve, V-cycle and solves, through the
C ABI against the oracle.  Tolerances as in test_gpu_parity."""
import numpy as np
import pytest
import torch

import paper_2411_14977_gb300.pmg as pmg
import workloads as W
from oracle import mg
from oracle.sem import apply_masked, relative_residual, solve_direct
from tests.gpu_helpers import Case, n, t

pytestmark = pytest.mark.gpu


def periodic_two_orders(cells_x=8, cells_z=2, order=7, order_z=8):
    L = 0.390625 * cells_x
    s = W.Surface(0.04, 2 * np.pi / L)
    return W.Workload(f"periodic_{cells_x}x{cells_z}_p{order}z{order_z}", cells_x, cells_z, order, 0.0, L, 1.0, True,
                      W.BASE_SEED + 95, s, "div", velocity=W.Velocity.random(W.BASE_SEED + 96), order_z=order_z)


def source_two_orders(cells_x=9, cells_z=2, order=3, order_z=8):
    w = W.config1()
    return W.Workload(f"source_{cells_x}x{cells_z}_p{order}z{order_z}", cells_x, cells_z, order, 0.0, 10.0, 1.0,
                      False, W.BASE_SEED + 97, W.Surface(0.05, 2 * np.pi / 10), "source",
                      pressure=w.pressure, noise_sd=1e-3, order_z=order_z)


CASES = {
    "p2z8": lambda: W.paper_scaling(12, 2, order_z=8),
    "p4z8": lambda: W.paper_scaling(10, 4, order_z=8),
    "p6z8": lambda: W.paper_scaling(8, 6, order_z=8),
    "p9z8": lambda: W.paper_scaling(6, 9, order_z=8),
    "p10z8": lambda: W.paper_scaling(5, 10, order_z=8),
    "p3z8_src": lambda: source_two_orders(),
    "p7z8_periodic": lambda: periodic_two_orders(),
    "p5z8_nz1": lambda: W.Workload("p5z8_nz1", 7, 1, 5, 0.0, 4.0, 1.0, False, W.BASE_SEED + 98,
                                   W.Surface(0.03, 2 * np.pi / 4), "div",
                                   velocity=W.Velocity.random(W.BASE_SEED + 99), order_z=8),
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
def test_apply_two_orders(name, df64):
    c = case(name, df64_outer=df64)
    assert c.m.Pz == 8 and c.S.NZ == c.m.NZ
    A = c.m.assemble(c.eta)
    x = np.random.default_rng(31).standard_normal(c.m.N)
    dm = c.m.dirichlet_mask()
    ref = apply_masked(A, x, dm)
    s = scale_of(A, np.where(dm, 0, x))
    assert np.max(np.abs(n(c.S.apply(t(x))) - ref)) <= 1e-12 * s
    assert np.max(np.abs(n(c.S.apply_f32(t(x, torch.float32))) - ref)) <= 2e-5 * s


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_two_orders(name):
    c = case(name)
    ref = c.rhs_oracle()
    assert np.max(np.abs(n(c.rhs_gpu()) - ref)) <= 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("flat", [0, 1])
@pytest.mark.parametrize("name", list(CASES))
def test_level_operators_and_transfers_two_orders(name, flat):
    c = case(name, flat_kernel=flat)
    H = c.hierarchy()
    assert [c.S.level_info(l)[0] for l in range(len(H.levels))] == H.orders
    assert [c.S.level_info(l)[2] for l in range(len(H.levels))] == [lev.mesh.NZ for lev in H.levels]
    rng = np.random.default_rng(32)
    for l, lev in enumerate(H.levels):
        N = lev.mesh.N
        x = rng.standard_normal(N)
        x[lev.dmask] = 0.0
        ref = lev.A @ x[lev.free]
        s = np.max(np.abs(lev.A) @ np.abs(x[lev.free]))
        for dt, tol in ((torch.float64, 1e-12), (torch.float32, 2e-5)):
            y = n(c.S.level_apply(l, t(x, dt)))
            assert np.max(np.abs(y[lev.free] - ref)) <= tol * s, (l, dt)
        if l == len(H.levels) - 1:
            continue
        C = H.levels[l + 1]
        rf = rng.standard_normal(N)
        rf[lev.dmask] = 0.0
        rc_ref = np.zeros(C.mesh.N)
        rc_ref[C.free] = H.P[l].T @ rf[lev.free]
        xc = rng.standard_normal(C.mesh.N)
        xc[C.dmask] = 0.0
        xf0 = rng.standard_normal(N)
        xf0[lev.dmask] = 0.0
        xf_ref = xf0.copy()
        xf_ref[lev.free] += H.P[l] @ xc[C.free]
        for dt, tol in ((torch.float64, 1e-13), (torch.float32, 1e-5)):
            rc = n(c.S.restrict(l, t(rf, dt), torch.zeros(C.mesh.N, dtype=dt, device="cuda")))
            assert np.max(np.abs(rc - rc_ref)) <= tol * max(1.0, np.max(np.abs(rc_ref))), (l, dt)
            xf = n(c.S.prolong(l, t(xc, dt), t(xf0, dt)))
            assert np.max(np.abs(xf - xf_ref)) <= tol * max(1.0, np.max(np.abs(xf_ref))), (l, dt)


@pytest.mark.parametrize("name", list(CASES))
def test_smoother_two_orders(name):
    c = case(name)
    H = c.hierarchy()
    rng = np.random.default_rng(33)
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
def test_coarse_solve_and_vcycle_two_orders(name):
    c = case(name)
    H = c.hierarchy()
    rng = np.random.default_rng(34)
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
            dict(precision=pmg.PMG_MIXED_FP32, flat_kernel=1)]


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("variant", VARIANTS)
def test_solve_two_orders(name, variant):
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
    if not variant:
        _, its, _, _ = mg.solve(c.m, c.eta, bo, c.F["pD"], tol=1e-12, overlap=1, nu=2, omega=0.8)
        assert abs(info["iterations"] - its) <= 1, (info["iterations"], its)


def test_autotune_two_orders():
    c = Case(W.paper_scaling(24, 4, order_z=8), tol=1e-11, precision=pmg.PMG_MIXED_FP32)
    c.S.autotune()
    bo = c.rhs_oracle()
    A = c.m.assemble(c.eta)
    dm = c.m.dirichlet_mask()
    pref = solve_direct(A, bo, c.F["pD"], dm)
    p, _ = c.S.solve(c.rhs_gpu(), t(c.F["pD"]))
    assert np.linalg.norm(n(p) - pref) / np.linalg.norm(pref) <= 1e-9


def test_two_orders_rejections():
    with pytest.raises(pmg.PmgError):
        pmg.Solver(6, 2, 3, order_z=6)                     # pair not built
    with pytest.raises(pmg.PmgError):
        pmg.Solver(6, 2, 4, order_z=8, nlevels=3, level_orders=[4, 2, 1])
    with pytest.raises(pmg.PmgError):
        pmg.Solver(6, 2, 4, order_z=8, precision=pmg.PMG_MIXED_BF16, outer=pmg.PMG_IR)
    c = case("p4z8")
    with pytest.raises(pmg.PmgError):
        c.S.set_bathymetry(torch.ones(c.S.NX, dtype=torch.float64, device="cuda"))
    with pytest.raises(pmg.PmgError):
        c.S.set_geometry_mixed(t(c.eta), t(c.eta))
    with pytest.raises(pmg.PmgError):
        c.S.gradient(torch.zeros(c.S.n, dtype=torch.float64, device="cuda"))
    # equal orders given explicitly are the default handle
    S = pmg.Solver(6, 2, 4, order_z=4)
    assert S.NZ == 2 * 4 + 1
    S.close()
