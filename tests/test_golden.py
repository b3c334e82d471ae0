"""The oracle's Runge-Kutta tableaux against the ones printed in Appendix D
(tests/golden/ssp_rk_tableaux.txt): the oracle must integrate with the
printed digits, and the printed tableaux must be the consistent SSP methods
the text says they are (rows summing to the nodes, weights summing to one to
the printed precision, order conditions to the printed precision)."""
import numpy as np
import pytest

import golden_values
from oracle import pyoracle as O

TABS = golden_values.rk_tableaux()


@pytest.mark.parametrize("order", [2, 3, 4])
def test_oracle_uses_the_printed_tableau(order):
    A, b, c = O.rk_tableau(order)
    gA, gb, gc = TABS[order]
    np.testing.assert_array_equal(A, gA)
    np.testing.assert_array_equal(b, gb)
    np.testing.assert_array_equal(c, gc)


@pytest.mark.parametrize("order", [2, 3, 4])
def test_printed_tableau_is_consistent(order):
    """Row sums equal the printed nodes and the classical order conditions
    up to the method's order hold, to the 14 printed digits."""
    A, b, c = TABS[order]
    np.testing.assert_allclose(A.sum(axis=1), c, atol=2e-14)
    conds = [(b.sum(), 1.0), (b @ c, 0.5)]
    if order >= 3:
        conds += [(b @ c ** 2, 1 / 3), (b @ A @ c, 1 / 6)]
    if order >= 4:
        conds += [(b @ c ** 3, 1 / 4), (b @ (c * (A @ c)), 1 / 8), (b @ A @ c ** 2, 1 / 12),
                  (b @ A @ A @ c, 1 / 24)]
    for got, want in conds:
        assert abs(got - want) < (1e-13 if order < 4 else 2e-10), (order, got, want)
    # a fifth-order condition fails for the fourth-order method (the check can fail)
    if order == 4:
        assert abs(b @ c ** 4 - 1 / 5) > 1e-4

