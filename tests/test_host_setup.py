"""The library's host-side setup against the oracle, without a GPU: the level orders that
pmg_create plans (Sec. 5.1 coarsening rule, semi-coarsening for two orders, a custom
list) and the reference-element tables (Sec. 4.3 LGL nodes and weights, the derivative
matrix; Sec. 5.2 the 1D interpolation factor of the prolongation).  The two sides are
separate implementations (C++ in the library, numpy in the oracle)."""
import numpy as np
import pytest

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
