"""Pins of the oracle's reference-element basis (Sec. 4.3, Sec. 5.1-5.2) against closed
forms and independent library routines (numpy.polynomial)."""
import numpy as np
import numpy.polynomial.legendre as npleg
import pytest

from oracle import basis

CLOSED_FORM_LGL = {
    1: ([-1.0, 1.0], [1.0, 1.0]),
    2: ([-1.0, 0.0, 1.0], [1 / 3, 4 / 3, 1 / 3]),
    3: ([-1.0, -1 / np.sqrt(5), 1 / np.sqrt(5), 1.0], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    4: ([-1.0, -np.sqrt(3 / 7), 0.0, np.sqrt(3 / 7), 1.0],
        [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
}


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lgl_closed_forms(p):
    x, w = basis.lgl_nodes_weights(p)
    xe, we = CLOSED_FORM_LGL[p]
    np.testing.assert_allclose(x, xe, atol=1e-15)
    np.testing.assert_allclose(w, we, atol=1e-15)


@pytest.mark.parametrize("p", range(1, 13))
def test_lgl_exactness_degree_2p_minus_1(p):
    x, w = basis.lgl_nodes_weights(p)
    for k in range(2 * p):
        exact = (1 - (-1) ** (k + 1)) / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-13


@pytest.mark.parametrize("n", [0, 1, 2, 5, 10])
def test_legendre_matches_numpy(n):
    x = np.linspace(-1, 1, 17)
    ours = basis.legendre_orthonormal(x, n)
    ours_d = basis.legendre_orthonormal_deriv(x, n)
    for k in range(n + 1):
        c = np.zeros(k + 1)
        c[k] = np.sqrt((2 * k + 1) / 2)
        np.testing.assert_allclose(ours[:, k], npleg.legval(x, c), atol=1e-13)
        np.testing.assert_allclose(ours_d[:, k], npleg.legval(x, npleg.legder(c)), atol=1e-11)


def test_orthonormal_by_gauss_legendre():
    xg, wg = npleg.leggauss(20)
    P = basis.legendre_orthonormal(xg, 10)
    np.testing.assert_allclose(P.T @ (wg[:, None] * P), np.eye(11), atol=1e-13)


@pytest.mark.parametrize("p", range(1, 11))
def test_exact_mass_rowsums_and_quadrature(p):
    M = basis.exact_mass_1d(p)
    _, w = basis.lgl_nodes_weights(p)
    np.testing.assert_allclose(M.sum(axis=1), w, atol=1e-13)
    # entries equal int h_i h_j by an independent Gauss rule of the Lagrange basis
    x, _ = basis.lgl_nodes_weights(p)
    xg, wg = npleg.leggauss(p + 2)
    H = np.zeros((xg.size, p + 1))
    for i in range(p + 1):
        others = np.delete(x, i)
        H[:, i] = np.prod((xg[:, None] - others[None, :]) / (x[i] - others[None, :]), axis=1)
    np.testing.assert_allclose(M, H.T @ (wg[:, None] * H), atol=1e-13)


@pytest.mark.parametrize("p", range(1, 11))
def test_diff_matrix_exact_on_polynomials(p):
    x, _ = basis.lgl_nodes_weights(p)
    D = basis.diff_matrix(p)
    for k in range(p + 1):
        expected = k * x ** (k - 1) if k > 0 else np.zeros_like(x)
        np.testing.assert_allclose(D @ x ** k, expected, atol=1e-11 * max(1, k * k))


@pytest.mark.parametrize("pc,pf", [(1, 2), (2, 3), (3, 4), (3, 5), (4, 6), (5, 8), (2, 8)])
def test_transfer_exact_on_coarse_polynomials(pc, pf):
    xc, _ = basis.lgl_nodes_weights(pc)
    xf, _ = basis.lgl_nodes_weights(pf)
    J = basis.transfer_1d(pc, pf)
    assert J.shape == (pf + 1, pc + 1)
    rng = np.random.default_rng(0)
    c = rng.standard_normal(pc + 1)
    np.testing.assert_allclose(J @ np.polyval(c, xc), np.polyval(c, xf), atol=1e-12)
    # end points are injections (continuity across elements)
    np.testing.assert_allclose(J[0], np.eye(pc + 1)[0], atol=1e-14)
    np.testing.assert_allclose(J[-1], np.eye(pc + 1)[-1], atol=1e-14)


def test_coarsening_rule():
    assert basis.coarsening_sequence(4) == [4, 3, 2, 1]
    assert basis.coarsening_sequence(5) == [5, 3, 2, 1]
    assert basis.coarsening_sequence(6) == [6, 4, 3, 2, 1]
    assert basis.coarsening_sequence(7) == [7, 4, 3, 2, 1]
    assert basis.coarsening_sequence(8) == [8, 5, 3, 2, 1]
    assert basis.coarsening_sequence(2) == [2, 1]
    assert basis.coarsening_sequence(1) == [1]
