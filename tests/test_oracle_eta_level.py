"""Pin of the oracle's level geometry: the surface (and the still-water depth) that each
multigrid level is built on (Sec. 5, Sec. 5.4: a level re-discretised on the current
geometry; Sec. 5.2: the level's nodal values are the fine interpolant evaluated at the
level's nodes, I = Phi V^-1).

The fine nodal values are samples of a continuous piecewise polynomial of degree <= P
per cell, so the fine interpolant IS that polynomial, and the level values must equal it
evaluated at the level's Legendre-Gauss-Lobatto nodes.  The expected values come from
numpy.polynomial (LGL nodes as +-1 and the roots of P_p', evaluation of the per-cell
polynomials), not from the oracle.  Sampling the nearest fine node, a linear
interpolation, or a transposed or mis-ordered transfer fails these checks.
"""
import numpy as np
import numpy.polynomial.legendre as npleg
import pytest
from numpy.polynomial import Polynomial

from oracle import basis
from oracle.mg import Hierarchy
from oracle.sem import Mesh


def lgl_numpy(p):
    """LGL nodes of order p on [-1, 1]: the end points and the roots of P_p'."""
    inner = npleg.Legendre.basis(p).deriv().roots() if p >= 2 else np.array([])
    return np.concatenate([[-1.0], np.sort(np.real(inner)), [1.0]])


class PiecewisePoly:
    """Continuous surface of degree <= P on each of Nx cells of [x0, x1] (periodic when
    asked): q_e(s) = a_e (1-s)/2 + a_{e+1} (1+s)/2 + (1 - s^2) r_e(s), r_e of degree P-2."""

    def __init__(self, Nx, P, x0, x1, periodic, seed, amp=0.05):
        rng = np.random.default_rng(seed)
        self.Nx, self.x0, self.dx = Nx, x0, (x1 - x0) / Nx
        a = amp * rng.standard_normal(Nx + 1)
        if periodic:
            a[-1] = a[0]
        self.a = a
        self.r = [Polynomial(amp * rng.standard_normal(max(P - 1, 1))) for _ in range(Nx)]

    def at(self, e, s):
        s = np.asarray(s, float)
        return self.a[e] * (1 - s) / 2 + self.a[e + 1] * (1 + s) / 2 + (1 - s * s) * self.r[e](s)

    def nodal(self, p, periodic):
        """Values at the node columns of an order-p mesh (column ex p + i, cell ex)."""
        s = lgl_numpy(p)
        NX = self.Nx * p + (0 if periodic else 1)
        out = np.empty(NX)
        for e in range(self.Nx):
            cols = e * p + np.arange(p + 1)
            v = self.at(e, s)
            if periodic:
                cols = cols % NX
            out[cols] = v
        return out


SEQ = {6: [6, 4, 3, 2, 1], 8: [8, 5, 3, 2, 1], 5: [5, 3, 2, 1]}


@pytest.mark.parametrize("P", [5, 6, 8])
@pytest.mark.parametrize("periodic", [False, True])
def test_eta_at_level_is_the_fine_polynomial_at_the_level_nodes(P, periodic):
    Nx, Nz = 8, 2
    q = PiecewisePoly(Nx, P, 0.0, 3.125, periodic, seed=100 + P)
    fine = Mesh(Nx, Nz, P, 0.0, 3.125, 1.0, periodic)
    # the oracle's node columns agree with the independent LGL nodes
    np.testing.assert_allclose(fine.column_x()[: P + 1], (lgl_numpy(P) + 1) / 2 * fine.dx, atol=1e-14)
    eta = q.nodal(P, periodic)
    assert basis.coarsening_sequence(P) == SEQ[P]
    gap = 0.0
    for p in SEQ[P][1:]:
        ml = Mesh(Nx, Nz, p, 0.0, 3.125, 1.0, periodic)
        got = Hierarchy._eta_at_level(fine, eta, ml)
        want = q.nodal(p, periodic)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)
        # sampling the nearest fine node instead (exact only where the level's nodes are
        # fine nodes, as at orders 1 and 2 for even P)
        xf, xl = fine.column_x(), ml.column_x()
        nearest = eta[np.abs(xl[:, None] - xf[None, :]).argmin(axis=1)]
        gap = max(gap, np.max(np.abs(nearest - want)))
    assert gap > 1e-3  # the check discriminates


@pytest.mark.parametrize("P", [6, 8])
def test_level_depth_is_the_fine_depth_polynomial(P):
    """A varying still-water depth reaches every level as the fine depth interpolant at
    the level's nodes (the flat level operator keeps each node column's depth)."""
    Nx, Nz = 6, 2
    q = PiecewisePoly(Nx, P, 0.0, 2.5, False, seed=7 + P, amp=0.1)
    depth = 0.6 + q.nodal(P, False)
    assert depth.min() > 0.2
    fine = Mesh(Nx, Nz, P, 0.0, 2.5, 1.0, False, depth=depth)
    H = Hierarchy(fine, np.zeros(fine.NX), overlap=1, nu=1, omega=0.8, geometry='flat')
    for lev, p in zip(H.levels, SEQ[P]):
        np.testing.assert_allclose(lev.mesh.hcol, 0.6 + q.nodal(p, False), rtol=0, atol=1e-13)


def test_actual_geometry_levels_use_the_level_surface():
    """geometry='actual': each level matrix equals the same-order mesh assembled on the
    fine surface polynomial evaluated at that level's nodes (expected values from
    numpy.polynomial); the order-1 level keeps the flat operator when asked."""
    P, Nx, Nz = 6, 5, 2
    q = PiecewisePoly(Nx, P, 0.0, 2.0, False, seed=31)
    fine = Mesh(Nx, Nz, P, 0.0, 2.0, 1.0, False)
    eta = q.nodal(P, False)
    H = Hierarchy(fine, eta, overlap=1, nu=1, omega=0.8, geometry='actual', coarse_geometry='flat')
    for l, (lev, p) in enumerate(zip(H.levels, SEQ[P])):
        ml = Mesh(Nx, Nz, p, 0.0, 2.0, 1.0, False)
        surf = np.zeros(ml.NX) if l == len(H.levels) - 1 else q.nodal(p, False)
        A = ml.assemble(surf).tocsr()[lev.free][:, lev.free]
        assert abs(A - lev.A).max() <= 1e-12 * abs(A).max()
        if 0 < l < len(H.levels) - 1:
            # and differs from the flat operator by far more (the surface matters)
            Af = ml.assemble(np.zeros(ml.NX)).tocsr()[lev.free][:, lev.free]
            assert abs(Af - lev.A).max() > 1e-4 * abs(A).max()
