"""The library's host-side setup against the oracle, without a GPU: the level orders that
pmg_create plans (Sec. 5.1 coarsening rule, semi-coarsening for two orders, a custom
list), the reference-element tables (Sec. 4.3 LGL nodes and weights, the derivative
matrix; Sec. 5.2 the 1D interpolation factor of the prolongation) and the fast-
diagonalisation factors of the Schwarz element classes (Sec. 5.3, against blocks built
here and scipy's generalized symmetric eigensolver).  The two sides are separate
implementations (C++ in the library; numpy and scipy here and in the oracle)."""
import numpy as np
import pytest
import scipy.linalg as sla

import paper_2411_14977_gb300.pmg as pmg
from oracle import basis


@pytest.mark.parametrize("P", range(2, 11))
def test_level_orders_follow_the_coarsening_rule(P):
    got = pmg.level_sequence(8, 2, P)
    assert got == [(p, p) for p in basis.coarsening_sequence(P)]


@pytest.mark.parametrize("P", range(2, 11))
def test_semi_coarsened_level_pairs(P):
    """Sec. 6.3's shape: P_z = 8 with every horizontal order 2..10."""
    got = pmg.level_sequence(200, 2, P, order_z=8)
    assert got == [tuple(pr) for pr in basis.semi_coarsening_sequence(P, 8)]


def test_custom_level_orders_and_their_checks():
    assert pmg.level_sequence(8, 2, 6, level_orders=[6, 3, 1]) == [(6, 6), (3, 3), (1, 1)]
    with pytest.raises(pmg.PmgError, match="decrease"):
        pmg.level_sequence(8, 2, 6, level_orders=[6, 6, 1])
    with pytest.raises(pmg.PmgError, match="order to 1"):
        pmg.level_sequence(8, 2, 6, level_orders=[6, 3])
    with pytest.raises(pmg.PmgError, match="order must be >= 2"):
        pmg.level_sequence(8, 2, 1)
    with pytest.raises(pmg.PmgError, match="equal orders"):
        pmg.level_sequence(8, 2, 6, order_z=8, level_orders=[6, 3, 1])


@pytest.mark.parametrize("p", range(1, 11))
def test_lgl_nodes_weights_and_derivative_matrix(p):
    t = pmg.basis_tables(p)
    x, w = basis.lgl_nodes_weights(p)
    np.testing.assert_allclose(t["nodes"].numpy(), x, rtol=0, atol=1e-14)
    np.testing.assert_allclose(t["weights"].numpy(), w, rtol=0, atol=1e-14)
    np.testing.assert_allclose(t["D"].numpy(), basis.diff_matrix(p), rtol=0, atol=2e-12 * p * p)
    assert t["J"] is None


@pytest.mark.parametrize("pc,p", [(1, 2), (1, 10), (2, 3), (3, 5), (4, 6), (5, 8), (6, 10), (7, 7)])
def test_prolongation_factor(pc, p):
    t = pmg.basis_tables(p, pc)
    np.testing.assert_allclose(t["J"].numpy(), basis.transfer_1d(pc, p), rtol=0, atol=1e-12)


@pytest.mark.parametrize("p,pc", [(0, 0), (11, 0), (4, 5), (4, -1)])
def test_basis_tables_reject_bad_orders(p, pc):
    with pytest.raises(pmg.PmgError):
        pmg.basis_tables(p, pc)


def _line_block(p, o, direction, cls):
    """The class's 1D subdomain block built here from its definition: assembled LGL
    stiffness sum_cells D^T diag(w) D and assembled weights on a canonical line, restricted
    to the element's node lines plus o lines each side (cut at the line's ends; along
    sigma the top node is Dirichlet)."""
    ncell = 3 if cls == 0 else (1 if cls == 3 else 2)
    e = 1 if cls in (0, 2) else 0
    n = ncell * p + 1
    D = basis.diff_matrix(p)
    _, w = basis.lgl_nodes_weights(p)
    K, M = np.zeros((n, n)), np.zeros(n)
    for c in range(ncell):
        idx = c * p + np.arange(p + 1)
        K[np.ix_(idx, idx)] += D.T @ np.diag(w) @ D
        M[idx] += w
    last = n - 1 - (1 if direction == 1 else 0)
    loc, glob = [], []
    for a in range(p + 1 + 2 * o):
        g = e * p - o + a
        if 0 <= g <= last:
            loc.append(a)
            glob.append(g)
    return K[np.ix_(glob, glob)], M[glob], loc


@pytest.mark.parametrize("p", [1, 2, 3, 4, 6, 8, 10])
@pytest.mark.parametrize("o", [0, 1])
@pytest.mark.parametrize("direction", [0, 1])
@pytest.mark.parametrize("cls", [0, 1, 2, 3])
def test_schwarz_class_factors_diagonalise_the_block(p, o, direction, cls):
    """V^T M V = I and V^T K V = diag(lam) on the block's nodes, the eigenvalues those of
    scipy's generalized symmetric solver, zero rows for absent nodes (Sec. 5.3)."""
    V, lam, k = pmg.schwarz_class(p, o, direction, cls)
    V, lam = V.numpy(), lam.numpy()
    K, M, loc = _line_block(p, o, direction, cls)
    assert k == len(loc)
    Vk = V[np.ix_(loc, range(k))]
    np.testing.assert_allclose(Vk.T @ np.diag(M) @ Vk, np.eye(k), atol=1e-11)
    scale = max(1.0, np.max(np.abs(lam)))
    np.testing.assert_allclose(Vk.T @ K @ Vk, np.diag(lam[:k]), atol=1e-10 * scale)
    ref = sla.eigh(K, np.diag(M), eigvals_only=True)
    np.testing.assert_allclose(np.sort(lam[:k]), ref, atol=1e-10 * scale)
    absent = [a for a in range(V.shape[0]) if a not in loc]
    assert np.all(V[absent] == 0.0) and np.all(V[:, k:] == 0.0) and np.all(lam[k:] == 0.0)


@pytest.mark.parametrize("args", [(0, 0, 0, 0), (11, 0, 0, 0), (4, 2, 0, 0), (4, 0, 2, 0), (4, 0, 0, 4)])
def test_schwarz_class_rejects_bad_arguments(args):
    with pytest.raises(pmg.PmgError):
        pmg.schwarz_class(*args)
