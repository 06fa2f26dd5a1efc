"""Pins of the oracle with different horizontal and vertical orders P_x != P_z (Sec. 5.1
semi-coarsening; Sec. 6.3 scaling study at N_z = 2, P_z = 8): closed-form level pairs, the
flat element as a Kronecker sum of 1D matrices of two orders, exact fluxes of linear
functions, spectral convergence in each order, exact transfers, and the hierarchy."""

import numpy as np
import pytest

from oracle import basis, mg
from oracle.sem import Mesh, solve_direct
import workloads as W


def test_semi_coarsening_sequences():
    f = basis.semi_coarsening_sequence
    assert f(4, 8) == [(4, 8), (4, 5), (4, 4), (3, 3), (2, 2), (1, 1)]
    assert f(2, 8) == [(2, 8), (2, 5), (2, 3), (2, 2), (1, 1)]
    assert f(7, 8) == [(7, 8), (7, 7), (4, 4), (3, 3), (2, 2), (1, 1)]
    assert f(10, 8) == [(10, 8), (8, 8), (5, 5), (3, 3), (2, 2), (1, 1)]
    assert f(8, 3) == [(8, 3), (5, 3), (3, 3), (2, 2), (1, 1)]
    assert f(6, 6) == [(p, p) for p in basis.coarsening_sequence(6)]


@pytest.mark.parametrize("P,Pz", [(2, 8), (5, 3), (8, 1)])
def test_flat_element_is_kronecker_sum_of_two_orders(P, Pz):
    """K_e = (h dsig/dx) S_x (x) W_z + (dx/(h dsig)) W_x (x) S_z, S = D^T M D with each
    direction's own order and exact mass (Sec. 4.3), W the LGL weights."""
    m = Mesh(3, 2, P, 0.0, 2.7, h=1.3, order_z=Pz)
    K = m.element_stiffness(np.zeros(m.NX), elems=[0])[0]
    Sx = basis.diff_matrix(P).T @ basis.exact_mass_1d(P) @ basis.diff_matrix(P)
    Sz = basis.diff_matrix(Pz).T @ basis.exact_mass_1d(Pz) @ basis.diff_matrix(Pz)
    _, wx = basis.lgl_nodes_weights(P)
    _, wz = basis.lgl_nodes_weights(Pz)
    cx = m.h * m.dsig / m.dx
    cz = m.dx / (m.h * m.dsig)
    np.testing.assert_allclose(K, cx * np.kron(Sx, np.diag(wz)) + cz * np.kron(np.diag(wx), Sz), atol=1e-12)


def _flux(m, eta, alpha, beta):
    """int_Gamma N_i (alpha, beta).n ds: top (-eta_x, 1) dx, flat bottom (0, -1) dx, walls
    (-+1, 0) d dsig/2, by numpy polynomial fits of the surface per cell."""
    out = np.zeros(m.N)
    xn = (m.r + 1) / 2 * m.dx
    for ex in range(m.Nx):
        cols = (ex * m.P + np.arange(m.P + 1)) % m.NX
        etax = np.polyval(np.polyder(np.polyfit(xn, eta[cols], m.P)), xn)
        for i in range(m.P + 1):
            out[cols[i] * m.NZ + m.NZ - 1] += m.w[i] * m.dx / 2 * (beta - alpha * etax[i])
            out[cols[i] * m.NZ] += m.w[i] * m.dx / 2 * (-beta)
    if not m.periodic:
        for ix, sgn in ((0, -1.0), (m.NX - 1, 1.0)):
            d = eta[ix] + m.h
            for ez in range(m.Nz):
                for j in range(m.Pz + 1):
                    out[ix * m.NZ + ez * m.Pz + j] += m.wz[j] * d * m.dsig / 2 * sgn * alpha
    return out


@pytest.mark.parametrize("P,Pz", [(2, 8), (6, 3), (1, 4), (9, 8)])
def test_linear_functions_exact_with_two_orders(P, Pz):
    m = Mesh(5, 2, P, 0.0, 3.0, h=1.0, order_z=Pz)
    x = m.column_x()
    eta = 0.07 * np.cos(2 * np.pi * x / 3.0) + 0.02 * np.sin(3.1 * x)
    A = m.assemble(eta)
    X, Z = m.node_xz(eta)
    for alpha, beta in ((1.0, 0.0), (0.0, 1.0), (0.7, -1.3)):
        np.testing.assert_allclose(A @ (alpha * X + beta * Z + 0.4), _flux(m, eta, alpha, beta), atol=1e-11)


def _harmonic_error(P, Pz):
    pf = W.Harmonic(2 * np.pi / 10, 0.3, 1.2)
    m = Mesh(10, 2, P, 0.0, 10.0, h=1.0, order_z=Pz)
    x = m.column_x()
    eta = 0.05 * np.cos(2 * np.pi * x / 10)
    X, Z = m.node_xz(eta)
    dm = m.dirichlet_mask()
    s = m.row_sigma()
    gb = -pf.grad(x, -np.ones(m.NX))[1]
    gl = -pf.grad(np.zeros(m.NZ), s * (eta[0] + 1) - 1)[0]
    gr = pf.grad(np.full(m.NZ, 10.0), s * (eta[-1] + 1) - 1)[0]
    b = m.rhs_source(eta, np.zeros(m.N), gb, gl, gr)
    p = solve_direct(m.assemble(eta), b, np.where(dm, pf(X, Z), 0.0), dm)
    return np.max(np.abs(p - pf(X, Z)))


def test_spectral_convergence_in_each_order():
    """Raising one order with the other fixed high reduces the error faster than
    algebraically until the fixed direction's error floor."""
    ex = np.array([_harmonic_error(P, 10) for P in range(2, 9)])
    ez = np.array([_harmonic_error(10, Pz) for Pz in range(2, 9)])
    for e in (ex, ez):
        above = e[e > 1e-12]                     # above the round-off floor
        assert above.size >= 4 and np.all(np.diff(above) < 0), e
        assert e[0] / e[4] > 1e3, e
    assert _harmonic_error(10, 10) < 1e-9


def test_prolongation_exact_on_coarse_polynomials():
    """A field of degree (p_x, p_z) per cell on the coarse level is prolonged exactly."""
    m = Mesh(4, 2, 3, 0.0, 2.0, h=1.0, order_z=8)
    H = mg.Hierarchy(m, np.zeros(m.NX), overlap=1)
    assert H.pairs == [(3, 8), (3, 5), (3, 3), (2, 2), (1, 1)]
    for l in range(len(H.levels) - 1):
        F, C = H.levels[l], H.levels[l + 1]
        Xc, Zc = C.mesh.node_xz(np.zeros(C.mesh.NX))
        Xf, Zf = F.mesh.node_xz(np.zeros(F.mesh.NX))
        px, pz = H.pairs[l + 1]
        f = lambda X, Z: (X ** px) * (Z ** pz) + 0.5 * X * Z
        # the field vanishes on the surface row z = 0, as the free-node transfer assumes
        np.testing.assert_allclose(H.P[l] @ f(Xc, Zc)[C.free], f(Xf, Zf)[F.free], atol=1e-11)


@pytest.mark.parametrize("P", [2, 4, 6, 10])
def test_hierarchy_two_orders_symmetric_and_converges(P):
    """Sec. 6.3 shape (N_z = 2, P_z = 8): PCG with the semi-coarsened V-cycle reaches the
    direct solution in a bounded number of iterations; the V-cycle is symmetric."""
    w = W.paper_scaling(20, P)
    m = Mesh(w.cells_x, 2, P, w.x0, w.x1, h=1.0, order_z=8)
    F = w.fields(m.column_x(), m.row_sigma())
    b = m.rhs_divergence(F["eta"], F["u"], F["w"])
    H = mg.Hierarchy(m, F["eta"], overlap=1, nu=2, omega=0.8)
    p, its, hist, _ = mg.solve(m, F["eta"], b, F["pD"], hier=H, tol=1e-10)
    pref = solve_direct(m.assemble(F["eta"]), b, F["pD"], m.dirichlet_mask())
    assert np.max(np.abs(p - pref)) < 1e-8 * np.max(np.abs(pref))
    assert its <= 14, its
    n = H.levels[0].free.size
    r1, r2 = np.sin(np.arange(n)), np.cos(0.37 * np.arange(n))
    assert abs(r2 @ H.vcycle(r1) - r1 @ H.vcycle(r2)) <= 1e-12 * abs(r2 @ H.vcycle(r1))


def test_iterations_flat_in_horizontal_order():
    """Sec. 6.3: at N_z = 2, P_z = 8 the iteration count varies very little with P_x."""
    its = []
    for P in range(2, 11):
        w = W.paper_scaling(20, P)
        m = Mesh(w.cells_x, 2, P, w.x0, w.x1, h=1.0, order_z=8)
        F = w.fields(m.column_x(), m.row_sigma())
        b = m.rhs_divergence(F["eta"], F["u"], F["w"])
        its.append(mg.solve(m, F["eta"], b, F["pD"], tol=1e-6, overlap=1, nu=2, omega=0.8)[1])
    assert max(its) - min(its) <= 2 and max(its) <= 8, its
