"""Pins of the oracle on a varying still-water depth h(x) (Sec. 2.2: sigma = (z + h(x))/d,
d = eta + h(x); the bar experiment of Sec. 6 runs over such a bottom) against identities
that fix every metric term, and of the separable level operator of the preconditioner."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import basis, mg
from oracle.sem import Mesh, solve_direct
import workloads as W


def _bump(x0, x1, amp=0.35, rel_w=0.15):
    xc, w = 0.5 * (x0 + x1), rel_w * (x1 - x0)
    return lambda x: 1.0 - amp * np.exp(-((np.asarray(x) - xc) / w) ** 2)


def _periodic_bottom(L):
    return lambda x: 0.9 + 0.2 * np.sin(2 * np.pi * np.asarray(x) / L) + 0.05 * np.cos(6 * np.pi * np.asarray(x) / L)


def _poly_slope(m, vals):
    """d/dx of each cell's interpolant of nodal column values, at the cell's nodes, by
    numpy polynomial fitting (independent of the oracle's differentiation matrix)."""
    out = np.zeros((m.Nx, m.P + 1))
    xn = (m.r + 1) / 2 * m.dx
    for ex in range(m.Nx):
        cols = (ex * m.P + np.arange(m.P + 1)) % m.NX
        c = np.polyfit(xn, vals[cols], m.P)
        out[ex] = np.polyval(np.polyder(c), xn)
    return out


def boundary_flux_linear(m, eta, alpha, beta):
    """int_Gamma N_i (alpha, beta).n ds per node by LGL edge quadrature: top n ds =
    (-eta_x, 1) dx, bottom z = -h(x): n ds = (-h_x, -1) dx, walls n ds = (-+1, 0) d dsig/2."""
    out = np.zeros(m.N)
    P, NZ = m.P, m.NZ
    etax = _poly_slope(m, eta)
    hx = _poly_slope(m, m.hcol)
    for ex in range(m.Nx):
        cols = (ex * P + np.arange(P + 1)) % m.NX
        for i in range(P + 1):
            ix = cols[i]
            out[ix * NZ + NZ - 1] += m.w[i] * m.dx / 2 * (beta - alpha * etax[ex, i])
            out[ix * NZ + 0] += m.w[i] * m.dx / 2 * (-beta - alpha * hx[ex, i])
    if not m.periodic:
        for ix, sgn in ((0, -1.0), (m.NX - 1, 1.0)):
            d = eta[ix] + m.hcol[ix]
            for ez in range(m.Nz):
                for j in range(P + 1):
                    out[ix * NZ + ez * P + j] += m.w[j] * d * m.dsig / 2 * sgn * alpha
    return out


def test_constant_depth_array_is_the_constant_depth_mesh():
    kw = dict(cells_x=5, cells_z=3, order=5, x0=0.0, x1=3.0, h=0.8)
    m0 = Mesh(**kw)
    m1 = Mesh(**kw, depth=np.full(m0.NX, 0.8))
    eta = 0.05 * np.cos(2.0 * m0.column_x())
    np.testing.assert_allclose(m1.assemble(eta).toarray(), m0.assemble(eta).toarray(), atol=1e-14)
    f = np.sin(np.arange(m0.N))
    gb = np.cos(np.arange(m0.NX))
    np.testing.assert_allclose(m1.rhs_source(eta, f, gb), m0.rhs_source(eta, f, gb), atol=1e-14)
    u, w = np.cos(np.arange(m0.N) * 0.3), np.sin(np.arange(m0.N) * 0.7)
    np.testing.assert_allclose(m1.rhs_divergence(eta, u, w), m0.rhs_divergence(eta, u, w), atol=1e-14)


@pytest.mark.parametrize("P,periodic", [(1, False), (2, False), (4, False), (6, True), (7, False)])
def test_linear_functions_exact_over_sloped_bottom(P, periodic):
    """a(N_i, l) for physical linear l = alpha x + beta z + c equals its boundary flux
    exactly: the pulled-back gradient of l is exact at the nodes (the cross metric term
    h_x - sigma d_x cancels the z-derivative of the map) and the remaining integrands are
    polynomials of degree <= 2P-1 in each direction.  A dropped or mis-signed h_x term
    fails the bottom rows."""
    L = 3.0
    depth = _periodic_bottom(L) if periodic else _bump(0.0, L)
    m = Mesh(5, 3, P, 0.0, L, h=1.0, periodic=periodic, depth=depth)
    x = m.column_x()
    eta = 0.07 * np.cos(2 * np.pi * x / L) + (0.0 if periodic else 0.02 * np.sin(3.1 * x))
    A = m.assemble(eta)
    X, Z = m.node_xz(eta)
    for alpha, beta in ((1.0, 0.0), (0.0, 1.0), (0.7, -1.3)):
        if periodic and alpha != 0.0:
            continue
        flux = boundary_flux_linear(m, eta, alpha, beta)
        np.testing.assert_allclose(A @ (alpha * X + beta * Z + 0.4), flux, atol=1e-11)


def test_divergence_rhs_equals_operator_on_gradients_over_sloped_bottom():
    m = Mesh(5, 3, 4, 0.0, 3.0, h=1.0, depth=_bump(0.0, 3.0))
    eta = 0.04 * np.cos(2.1 * m.column_x())
    A = m.assemble(eta)
    X, Z = m.node_xz(eta)
    b = m.rhs_divergence(eta, 0.6 * np.ones(m.N), -1.1 * np.ones(m.N))
    free = ~m.dirichlet_mask()
    np.testing.assert_allclose(b[free], (A @ (0.6 * X - 1.1 * Z))[free], atol=1e-12)


def test_symmetric_spd_and_neumann_nullspace_over_bar():
    wl = W.bar(12, 2, 5)
    m = Mesh(**wl.mesh_kwargs(), depth=wl.bathymetry)
    eta = wl.surface(m.column_x())
    Ad = m.assemble(eta).toarray()
    assert np.max(np.abs(Ad - Ad.T)) <= 1e-14 * np.max(np.abs(Ad))
    np.testing.assert_allclose(Ad @ np.ones(m.N), 0.0, atol=1e-12)
    free = ~m.dirichlet_mask()
    sla.cholesky(Ad[np.ix_(free, free)])


def test_spectral_convergence_over_bump():
    """p = cos(k (x + 0.3)) cosh(k (z + 1.2)) in a tank over a smooth bump: Dirichlet data on the
    surface, the exact normal derivative on the sloped bottom (n = -(h_x, 1)/|.|) and the
    walls.  The nodal error falls faster than algebraically in P."""
    k = 2 * np.pi / 10
    pfun = W.Harmonic(k, 0.3, 1.2)
    bump = W.Bar(1.0, 0.7, 3.5, 6.5, 1.0, 1.0)
    errs = []
    for P in range(2, 11):
        m = Mesh(12, 3, P, 0.0, 10.0, h=1.0, depth=bump)
        x = m.column_x()
        eta = 0.05 * np.cos(2 * np.pi * x / 10)
        X, Z = m.node_xz(eta)
        dmask = m.dirichlet_mask()
        pD = np.where(dmask, pfun(X, Z), 0.0)
        px, pz = pfun.grad(x, -m.hcol)
        hx = bump.slope(x)
        gb = -(hx * px + pz) / np.sqrt(1 + hx * hx)
        s = m.row_sigma()
        gl = -pfun.grad(np.full(m.NZ, 0.0), s * (eta[0] + m.hcol[0]) - m.hcol[0])[0]
        gr = pfun.grad(np.full(m.NZ, 10.0), s * (eta[-1] + m.hcol[-1]) - m.hcol[-1])[0]
        b = m.rhs_source(eta, np.zeros(m.N), gb, gl, gr)
        p = solve_direct(m.assemble(eta), b, pD, dmask)
        errs.append(np.max(np.abs(p - pfun(X, Z))))
    errs = np.array(errs)                        # P = 2 .. 10
    assert errs[-1] < 1e-10, errs
    assert np.all(np.diff(errs) < 0), errs
    # about a decade per order throughout: the reduction over P = 6 -> 10 is no smaller
    # than over P = 2 -> 6 (a fixed algebraic order would slow down)
    assert errs[0] / errs[4] > 1e3 and errs[4] / errs[8] > 1e3, errs


def test_separable_operator_constant_depth_is_flat_operator():
    m = Mesh(4, 3, 5, 0.0, 2.0, h=0.7)
    np.testing.assert_allclose(m.assemble_separable(m.hcol).toarray(),
                               m.assemble(np.zeros(m.NX)).toarray(), atol=1e-13)


@pytest.mark.parametrize("periodic", [False, True])
def test_separable_operator_is_kronecker_sum(periodic):
    """The slope-free level operator equals (dsig/dx) K_x[d] (x) M_z + (dx/dsig) M_x[1/d] (x) K_z
    with 1D matrices assembled here by numpy: K_x[d] from per-cell D^T diag(w d) D, M_x[1/d]
    the lumped weights over d, K_z, M_z the plain 1D LGL stiffness and weights."""
    P, Nx, Nz = 4, 5, 3
    L = 2.5
    m = Mesh(Nx, Nz, P, 0.0, L, h=1.0, periodic=periodic,
             depth=_periodic_bottom(L) if periodic else _bump(0.0, L))
    d = m.hcol
    D = basis.diff_matrix(P)
    w = m.w
    NX, NZ = m.NX, m.NZ
    Kx, Mx = np.zeros((NX, NX)), np.zeros(NX)
    for ex in range(Nx):
        cols = (ex * P + np.arange(P + 1)) % NX
        Kx[np.ix_(cols, cols)] += D.T @ np.diag(w * d[cols]) @ D
        Mx[cols] += w / d[cols]
    Kz, Mz = np.zeros((NZ, NZ)), np.zeros(NZ)
    for ez in range(Nz):
        rows = ez * P + np.arange(P + 1)
        Kz[np.ix_(rows, rows)] += D.T @ np.diag(w) @ D
        Mz[rows] += w
    ref = (m.dsig / m.dx) * np.kron(Kx, np.diag(Mz)) + (m.dx / m.dsig) * np.kron(np.diag(Mx), Kz)
    A = m.assemble_separable(d).toarray()
    np.testing.assert_allclose(A, ref, atol=1e-12 * np.max(np.abs(ref)))
    free = ~m.dirichlet_mask()
    sla.cholesky(A[np.ix_(free, free)])


def test_pmg_pcg_over_bar_matches_direct_solve():
    """The flat (slope-free, nodal depth) hierarchy preconditions the bar problem: PCG
    reaches the direct solution, in few iterations, and the V-cycle is symmetric."""
    wl = W.bar(16, 2, 6, rhs='source')
    m = Mesh(**wl.mesh_kwargs(), depth=wl.bathymetry)
    F = wl.fields(m.column_x(), m.row_sigma())
    eta = F['eta']
    b = m.rhs_source(eta, F['f'], F['g_bottom'], F['g_left'], F['g_right'])
    A = m.assemble(eta)
    dmask = m.dirichlet_mask()
    p_ref = solve_direct(A, b, F['pD'], dmask)
    hier = mg.Hierarchy(m, eta, overlap=1, nu=2, omega=0.8)
    assert hier.orders == [6, 4, 3, 2, 1]
    p, its, hist, _ = mg.solve(m, eta, b, F['pD'], hier=hier, method='pcg', tol=1e-10)
    assert its <= 20, its
    assert np.max(np.abs(p - p_ref)) < 1e-8 * np.max(np.abs(p_ref))
    n = hier.levels[0].free.size
    r1, r2 = np.sin(np.arange(n)), np.cos(0.37 * np.arange(n))
    z1, z2 = hier.vcycle(r1), hier.vcycle(r2)
    assert abs(r2 @ z1 - r1 @ z2) <= 1e-12 * abs(r2 @ z1)
