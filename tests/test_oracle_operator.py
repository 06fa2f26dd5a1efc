"""Pins of the oracle's sigma-mapped SEM operator, load vectors and direct solves
(Sec. 2.2, Sec. 3.2, Sec. 4.2-4.3) against closed forms, exact identities and brute force."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import basis
from oracle.sem import Mesh, solve_dense, solve_direct, relative_residual, apply_masked
import workloads as W


def curved_eta(m, amp=0.08, k=2 * np.pi / 3.0):
    return amp * np.cos(k * m.column_x()) + 0.3 * amp * np.sin(2.3 * k * m.column_x())


def test_flat_element_matches_exact_mass_construction():
    """Flat element: K_e = (h dsig/dx)(D^T M D) (x) W + (dx/(h dsig)) W (x) (D^T M D) with the
    exact 1D mass M = (V V^T)^-1 of Sec. 4.3 in the differentiated direction (LGL quadrature
    is exact there, degree 2P-2), lumped weights W in the other."""
    for P in (1, 3, 6, 8):
        m = Mesh(3, 2, P, 0.0, 2.7, h=1.3)
        K = m.element_stiffness(np.zeros(m.NX), elems=[0])[0]
        M = basis.exact_mass_1d(P)
        D = basis.diff_matrix(P)
        Wd = np.diag(m.w)
        S = D.T @ M @ D
        cx = m.h * m.dsig / m.dx
        cz = m.dx / (m.h * m.dsig)
        np.testing.assert_allclose(K, cx * np.kron(S, Wd) + cz * np.kron(Wd, S), atol=1e-12)


def _interp_poly(xn, vals):
    """Polynomial through (xn, vals) by numpy (independent of the oracle basis)."""
    return np.polyfit(xn, vals, len(xn) - 1)


def boundary_flux_linear(m, eta, alpha, beta):
    """int_Gamma N_i (alpha, beta).n ds for every node, by LGL edge quadrature written with
    numpy.polynomial (top: n ds = (-eta_x, 1) dx on the curved surface)."""
    out = np.zeros(m.N)
    P, NZ = m.P, m.NZ
    xn = (m.r + 1) / 2 * m.dx
    for ex in range(m.Nx):
        cols = ex * P + np.arange(P + 1)
        cols_w = cols % m.NX
        c = _interp_poly(xn, eta[cols_w])
        etax = np.polyval(np.polyder(c), xn)
        for i in range(P + 1):
            ix = cols_w[i]
            out[ix * NZ + NZ - 1] += m.w[i] * m.dx / 2 * (beta - alpha * etax[i])     # top
            out[ix * NZ + 0] += m.w[i] * m.dx / 2 * (-beta)                             # bottom
    if not m.periodic:
        for side, ix, sgn in ((0, 0, -1.0), (1, m.NX - 1, 1.0)):
            d = eta[ix] + m.h
            for ez in range(m.Nz):
                for j in range(P + 1):
                    out[ix * NZ + ez * P + j] += m.w[j] * d * m.dsig / 2 * sgn * alpha
    return out


@pytest.mark.parametrize("P,periodic", [(1, False), (2, False), (4, False), (6, True), (7, False)])
def test_linear_functions_exact_on_curved_mesh(P, periodic):
    """a(N_i, l) for physical linear l = alpha x + beta z + c equals the boundary flux exactly:
    LGL collocation integrates these (polynomial) integrands exactly on the sigma-map."""
    m = Mesh(5, 3, P, 0.0, 3.0, h=1.0, periodic=periodic)
    eta = curved_eta(m) if not periodic else 0.07 * np.cos(2 * np.pi * m.column_x() / 3.0)
    A = m.assemble(eta)
    X, Z = m.node_xz(eta)
    for alpha, beta in ((1.0, 0.0), (0.0, 1.0), (0.7, -1.3)):
        if periodic and alpha != 0.0:
            continue                        # x is not a periodic function
        lin = alpha * X + beta * Z + 0.4
        flux = boundary_flux_linear(m, eta, alpha, beta)
        np.testing.assert_allclose(A @ lin, flux, atol=1e-11)


def test_symmetric_spd_and_neumann_nullspace():
    m = Mesh(4, 3, 5, 0.0, 2.0, h=0.8)
    eta = curved_eta(m)
    A = m.assemble(eta)
    Ad = A.toarray()
    assert np.max(np.abs(Ad - Ad.T)) <= 1e-14 * np.max(np.abs(Ad))
    np.testing.assert_allclose(Ad @ np.ones(m.N), 0.0, atol=1e-12)
    free = ~m.dirichlet_mask()
    sla.cholesky(Ad[np.ix_(free, free)])          # raises if not SPD
    ev = np.linalg.eigvalsh(Ad)
    assert ev[0] > -1e-12 and ev[1] > 1e-8         # one-dimensional null space (constants)


def _solve_harmonic(m, eta, pfun, source=True):
    X, Z = m.node_xz(eta)
    dmask = m.dirichlet_mask()
    pD = np.where(dmask, pfun(X, Z), 0.0)
    xcol = m.column_x()
    s = m.row_sigma()
    gb = -pfun.grad(xcol, -m.h * np.ones(m.NX))[1]
    gl = -pfun.grad(np.full(m.NZ, m.x0), s * (eta[0] + m.h) - m.h)[0]
    gr = pfun.grad(np.full(m.NZ, m.x1), s * (eta[-1] + m.h) - m.h)[0]
    b = m.rhs_source(eta, np.zeros(m.N), gb, gl, gr)
    A = m.assemble(eta)
    return solve_direct(A, b, pD, dmask), pfun(X, Z)


@pytest.mark.parametrize("shift", [(0.0, 1.0), (0.3, 1.2)])
@pytest.mark.parametrize("curved", [False, True])
def test_spectral_convergence_to_harmonic(shift, curved):
    """Nodal max error to p = cos(k(x+xs))cosh(k(z+zs)) falls spectrally in P (Sec. 6.1 claims
    spectral p-convergence); (0.3, 1.2) has nonzero Neumann fluxes on all three sides."""
    pfun = W.Harmonic(2 * np.pi / 10, *shift)
    errs = []
    for P in range(1, 11):
        m = Mesh(16, 4, P, 0.0, 10.0, h=1.0)
        eta = 0.05 * np.cos(2 * np.pi * m.column_x() / 10) if curved else np.zeros(m.NX)
        p, pe = _solve_harmonic(m, eta, pfun)
        errs.append(np.max(np.abs(p - pe)))
    errs = np.array(errs)
    assert np.max(errs[7:]) < 1e-9, errs          # at the roundoff floor by P = 8
    above = errs[errs > 1e-11]
    assert above.size >= 4 and np.all(np.diff(above) < 0), errs
    # faster than algebraic: the error reduction per step in P does not stall
    ratios = above[1:] / above[:-1]
    assert np.all(ratios < 0.1), errs


def test_source_rhs_integrates_area_and_bottom_length():
    m = Mesh(6, 2, 5, 0.0, 3.0, h=1.0)
    eta = curved_eta(m)
    b = m.rhs_source(eta, np.ones(m.N))
    # area under the interpolated surface, by numpy polynomial integration per cell
    xn = (m.r + 1) / 2 * m.dx
    area = 0.0
    for ex in range(m.Nx):
        c = np.polyint(_interp_poly(xn, eta[ex * m.P + np.arange(m.P + 1)] + m.h))
        area += np.polyval(c, m.dx) - np.polyval(c, 0.0)
    free = ~m.dirichlet_mask()
    # top-row (Dirichlet) entries are zeroed, so compare against the unmasked sum
    rx, rz, sx, sz, J = m.element_metrics(eta)
    total = np.sum(m.quad_weights()[None, :] * J.reshape(J.shape[0], -1))
    assert abs(total - area) < 1e-12
    assert np.all(b[~free] == 0.0)
    gb = m.rhs_source(eta, np.zeros(m.N), g_bottom=np.ones(m.NX))
    assert abs(gb.sum() - 3.0) < 1e-13


def test_divergence_rhs_equals_operator_on_gradients():
    """b_div(grad q) = A q for physical linear q (both exact), all non-Dirichlet rows."""
    m = Mesh(5, 3, 4, 0.0, 3.0, h=1.0)
    eta = curved_eta(m)
    A = m.assemble(eta)
    X, Z = m.node_xz(eta)
    q = 0.6 * X - 1.1 * Z
    b = m.rhs_divergence(eta, 0.6 * np.ones(m.N), -1.1 * np.ones(m.N))
    free = ~m.dirichlet_mask()
    np.testing.assert_allclose(b[free], (A @ q)[free], atol=1e-12)


@pytest.mark.parametrize("wl", ["cfg1", "curved_small"])
def test_dense_bruteforce_equals_sparse_direct(wl):
    if wl == "cfg1":
        w = W.config1()
    else:
        w = W.tank(12, 3, 5)
    m = Mesh(**w.mesh_kwargs())
    F = w.fields(m.column_x(), m.row_sigma())
    eta = F['eta']
    if w.rhs == 'div':
        b = m.rhs_divergence(eta, F['u'], F['w'])
    else:
        b = m.rhs_source(eta, F['f'], F['g_bottom'], F['g_left'], F['g_right'])
    A = m.assemble(eta)
    dm = m.dirichlet_mask()
    p1 = solve_dense(A, b, F['pD'], dm)
    p2 = solve_direct(A, b, F['pD'], dm)
    assert np.linalg.norm(p1 - p2) <= 1e-12 * np.linalg.norm(p1)
    assert relative_residual(A, b, p1, dm) < 1e-13
    y = apply_masked(A, p1, dm)
    np.testing.assert_array_equal(y[dm], p1[dm])


def _two_surfaces(m):
    x = m.column_x()
    L = m.x1 - m.x0
    eta_k = 0.08 * np.cos(2 * np.pi * x / L) + 0.02 * np.sin(6 * np.pi * x / L)
    eta_km1 = 0.08 * np.cos(2 * np.pi * (x - 0.05) / L) + 0.03 * np.sin(6 * np.pi * x / L + 0.3)
    return eta_k, eta_km1


def test_mixed_stage_operator_reduces_to_same_stage():
    m = Mesh(cells_x=4, cells_z=2, order=4, x0=0.0, x1=2.0, h=1.0)
    eta_k, _ = _two_surfaces(m)
    Am = m.assemble_mixed(eta_k, eta_k).toarray()
    A = m.assemble(eta_k).toarray()
    np.testing.assert_allclose(Am, A, rtol=0, atol=1e-12 * np.abs(A).max())


@pytest.mark.parametrize("periodic", [False, True])
def test_mixed_stage_operator_on_physical_linear_functions(periodic):
    """A linear function of the physical coordinates has the same constant gradient on
    both stages' meshes, so A_mix(eta_k, eta_km1) l(stage k-1 nodes) = A(eta_k) l(stage k
    nodes) -- tying the mixed operator to the pinned same-stage one; and A_mix is not
    symmetric when the surfaces differ."""
    m = Mesh(cells_x=4, cells_z=3, order=5, x0=0.0, x1=2.0, h=1.0, periodic=periodic)
    eta_k, eta_km1 = _two_surfaces(m)
    Am = m.assemble_mixed(eta_k, eta_km1)
    A = m.assemble(eta_k)
    for al, be, ga in [(0.0, 0.0, 1.0), (0.0, 1.0, -0.3), (1.3, -0.7, 0.2)]:
        if periodic and al != 0.0:
            continue  # x is not periodic
        Xm, Zm = m.node_xz(eta_km1)
        Xk, Zk = m.node_xz(eta_k)
        lm = al * Xm + be * Zm + ga
        lk = al * Xk + be * Zk + ga
        np.testing.assert_allclose(Am @ lm, A @ lk, rtol=0, atol=1e-11 * max(1.0, np.abs(A @ lk).max()))
    D = (Am - Am.T).toarray()
    assert np.abs(D).max() > 1e-6 * np.abs(Am).max()
