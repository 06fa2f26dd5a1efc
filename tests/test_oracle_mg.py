"""Pins of the oracle's geometric p-multigrid (Sec. 5): transfers exact on coarse
polynomials, Schwarz exact in the one-subdomain limit, symmetric positive V-cycle,
Krylov answers equal to the direct solve, and flat iteration counts in N_x and P (Sec. 6.3)."""
import numpy as np
import pytest

from oracle import mg
from oracle.sem import Mesh, solve_direct
import workloads as W

DEFAULTS = dict(overlap=1, nu=2, omega=0.8)


def _problem(w):
    m = Mesh(**w.mesh_kwargs())
    F = w.fields(m.column_x(), m.row_sigma())
    eta = F['eta']
    if w.rhs == 'div':
        b = m.rhs_divergence(eta, F['u'], F['w'])
    else:
        b = m.rhs_source(eta, F['f'], F['g_bottom'], F['g_left'], F['g_right'])
    return m, eta, b, F['pD']


@pytest.mark.parametrize("pf", [2, 4, 6, 8])
def test_prolongation_exact_on_coarse_polynomials(pf):
    m = Mesh(3, 2, pf, 0.0, 2.0, h=1.0)
    H = mg.Hierarchy(m, np.zeros(m.NX), **DEFAULTS)
    for l in range(len(H.orders) - 1):
        fine, coarse = H.levels[l], H.levels[l + 1]
        pc = coarse.mesh.P

        def f(mesh):
            X, Z = mesh.node_xz(np.zeros(mesh.NX))
            # vanishes on the free surface z = 0; degree <= pc in x and in z
            return Z * (0.3 + X ** (pc) - 0.5 * X) * (1 + Z) ** (pc - 1)
        vf = f(fine.mesh)[fine.free]
        vc = f(coarse.mesh)[coarse.free]
        np.testing.assert_allclose(H.P[l] @ vc, vf, atol=1e-12)


@pytest.mark.parametrize("overlap", [0, 1, 2])
def test_schwarz_exact_for_one_subdomain(overlap):
    m = Mesh(1, 1, 5, 0.0, 1.0, h=1.0)
    H = mg.Hierarchy(m, np.zeros(m.NX), overlap=overlap, nu=1, omega=1.0)
    lev = H.levels[0]
    assert np.all(lev.W == 1.0)
    rng = np.random.default_rng(1)
    b = rng.standard_normal(lev.free.size)
    x = H.smooth(0, b, np.zeros_like(b), post=False)
    np.testing.assert_allclose(lev.A @ x, b, atol=1e-12)


def test_cover_counts_overlap_one():
    m = Mesh(3, 2, 4, 0.0, 3.0, h=1.0)
    H = mg.Hierarchy(m, np.zeros(m.NX), **DEFAULTS)
    lev = H.levels[0]
    cnt = 1.0 / lev.W
    P, NZ = 4, m.NZ

    def c1(i, n):      # 1D cover count of node line i with overlap 1 over n elements
        return sum(1 for e in range(n) if e * P - 1 <= i <= e * P + P + 1)
    for g, c in zip(lev.free, cnt):
        ix, iz = divmod(g, NZ)
        assert c == c1(ix, 3) * c1(iz, 2)


def test_vcycle_symmetric_positive():
    w = W.tank(6, 3, 6)
    m, eta, b, pD = _problem(w)
    for geom in ('flat', 'actual'):
        H = mg.Hierarchy(m, eta, geometry=geom, **DEFAULTS)
        n = H.levels[0].free.size
        rng = np.random.default_rng(2)
        for _ in range(3):
            u, v = rng.standard_normal(n), rng.standard_normal(n)
            Bu, Bv = H.vcycle(u), H.vcycle(v)
            assert abs(u @ Bv - v @ Bu) <= 1e-11 * abs(u @ Bv)
            assert v @ Bv > 0 and u @ Bu > 0


@pytest.mark.parametrize("method", ["pcg", "fcg", "pdc"])
def test_krylov_equals_direct(method):
    w = W.config1()
    m, eta, b, pD = _problem(w)
    p, its, hist, H = mg.solve(m, eta, b, pD, method=method, tol=1e-13, **DEFAULTS)
    pref = solve_direct(m.assemble(eta), b, pD, m.dirichlet_mask())
    assert np.linalg.norm(p - pref) <= 1e-11 * np.linalg.norm(pref)
    assert hist[-1] <= 1e-13


def test_curved_krylov_equals_direct_with_flat_preconditioner():
    w = W.tank(10, 4, 6)
    m, eta, b, pD = _problem(w)
    p, its, hist, H = mg.solve(m, eta, b, pD, tol=1e-13, geometry='flat', **DEFAULTS)
    pref = solve_direct(m.assemble(eta), b, pD, m.dirichlet_mask())
    assert np.linalg.norm(p - pref) <= 1e-11 * np.linalg.norm(pref)
    assert its < 40


def test_iterations_flat_in_nx_and_p():
    """Sec. 6.3: iteration counts show no tendency to grow with N_x (P = 8) or with P."""
    its_nx = []
    for nx in (8, 16, 32, 64):
        w = W.tank(nx, 2, 8)
        m, eta, b, pD = _problem(w)
        its_nx.append(mg.solve(m, eta, b, pD, tol=1e-6, **DEFAULTS)[1])
    # no growth with the number of degrees of freedom (one iteration of slack)
    assert all(b <= a + 1 for a, b in zip(its_nx, its_nx[1:])), its_nx
    assert its_nx[-1] <= its_nx[0], its_nx
    its_p = []
    for P in (4, 5, 6, 7, 8):
        w = W.tank(16, 2, P)
        m, eta, b, pD = _problem(w)
        its_p.append(mg.solve(m, eta, b, pD, tol=1e-6, **DEFAULTS)[1])
    assert max(its_p) - min(its_p) <= 3 and its_p[-1] <= its_p[0] + 2, its_p


def test_fgmres_finite_termination_and_scipy():
    """GMRES on an n x n system reaches the solution within n iterations (identity
    preconditioner, no restart); with the exact inverse as preconditioner in one; the
    result agrees with scipy.sparse.linalg.gmres; the residual history never increases
    within a cycle."""
    import scipy.sparse.linalg as spla
    rng = np.random.default_rng(7)
    n = 12
    A = rng.standard_normal((n, n)) + n * np.eye(n)  # nonsymmetric, well conditioned
    b = rng.standard_normal(n)
    x, its, hist = mg.fgmres(A, b, lambda v: v, tol=1e-13, restart=n)
    assert its <= n
    np.testing.assert_allclose(A @ x, b, atol=1e-11 * np.linalg.norm(b))
    assert all(h2 <= h1 * (1 + 1e-12) for h1, h2 in zip(hist[:-1], hist[1:-1]))
    Ainv = np.linalg.inv(A)
    x1, its1, _ = mg.fgmres(A, b, lambda v: Ainv @ v, tol=1e-12)
    assert its1 == 1
    xs, info = spla.gmres(A, b, rtol=1e-13, restart=n, atol=0.0)
    assert info == 0
    np.testing.assert_allclose(x, xs, rtol=0, atol=1e-10 * np.linalg.norm(xs))
    # restarted: still converges, more iterations than the unrestarted run
    x3, its3, _ = mg.fgmres(A, b, lambda v: v, tol=1e-10, restart=3)
    np.testing.assert_allclose(A @ x3, b, atol=1e-9 * np.linalg.norm(b))
    assert its3 >= its - 1


def test_fgmres_with_vcycle_matches_pcg_solution():
    w = W.tank(6, 2, 4)
    m = Mesh(**w.mesh_kwargs())
    F = w.fields(m.column_x(), m.row_sigma())
    b = m.rhs_divergence(F["eta"], F["u"], F["w"])
    p1, its_g, hist_g, _ = mg.solve(m, F["eta"], b, F["pD"], method="gmres", tol=1e-12, overlap=1, nu=2, omega=0.8)
    p2, its_c, _, _ = mg.solve(m, F["eta"], b, F["pD"], method="pcg", tol=1e-12, overlap=1, nu=2, omega=0.8)
    np.testing.assert_allclose(p1, p2, rtol=0, atol=1e-9 * np.abs(p2).max())
    assert hist_g[-1] <= 1e-12
    assert its_g <= its_c + 1


def test_actual_geometry_hierarchy_reduces_to_flat_at_rest_and_is_symmetric():
    """Re-discretised levels (geometry='actual', the coarsest kept flat): at eta = 0 the
    V-cycle is the flat one; on a wave it stays a symmetric preconditioner and PCG reaches
    the direct solution."""
    import workloads as W
    from oracle.sem import Mesh, solve_direct
    wl = W.tank(8, 2, 5)
    m = Mesh(**wl.mesh_kwargs())
    F = wl.fields(m.column_x(), m.row_sigma())
    flat = mg.Hierarchy(m, F["eta"], overlap=1, nu=2, omega=0.8)
    act0 = mg.Hierarchy(m, np.zeros(m.NX), overlap=1, nu=2, omega=0.8, geometry='actual', coarse_geometry='flat')
    n = flat.levels[0].free.size
    r = np.sin(np.arange(n) * 0.7)
    np.testing.assert_allclose(act0.vcycle(r), flat.vcycle(r), rtol=0, atol=1e-12 * np.abs(flat.vcycle(r)).max())
    eta = 4.0 * F["eta"]
    act = mg.Hierarchy(m, eta, overlap=1, nu=2, omega=0.8, geometry='actual', coarse_geometry='flat')
    r2 = np.cos(np.arange(n) * 0.3)
    assert abs(r2 @ act.vcycle(r) - r @ act.vcycle(r2)) <= 1e-12 * abs(r2 @ act.vcycle(r))
    b = m.rhs_divergence(eta, F["u"], F["w"])
    p, its, _, _ = mg.solve(m, eta, b, F["pD"], hier=act, tol=1e-10)
    pref = solve_direct(m.assemble(eta), b, F["pD"], m.dirichlet_mask())
    assert np.max(np.abs(p - pref)) <= 1e-8 * np.max(np.abs(pref)) and its <= 15
