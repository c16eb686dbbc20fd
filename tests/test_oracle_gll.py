"""Pins of the oracle's GLL tables against textbook values and exactness properties."""
import math

import numpy as np
import pytest
from numpy.polynomial import Polynomial

from oracle.gll import gll_nodes_weights, lagrange_derivative_matrix, lagrange_eval

# Textbook GLL rules (Abramowitz & Stegun 25.4.32 / any spectral-element text).
KNOWN = {
    1: ([-1.0, 1.0], [1.0, 1.0]),
    2: ([-1.0, 0.0, 1.0], [1 / 3, 4 / 3, 1 / 3]),
    3: ([-1.0, -1 / math.sqrt(5), 1 / math.sqrt(5), 1.0], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
    4: ([-1.0, -math.sqrt(3 / 7), 0.0, math.sqrt(3 / 7), 1.0], [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
}


@pytest.mark.parametrize("k", sorted(KNOWN))
def test_known_rules(k):
    x, w = gll_nodes_weights(k)
    np.testing.assert_allclose(x, KNOWN[k][0], atol=1e-15)
    np.testing.assert_allclose(w, KNOWN[k][1], rtol=1e-14)


@pytest.mark.parametrize("k", range(1, 9))
def test_quadrature_exact_to_degree_2k_minus_1(k):
    x, w = gll_nodes_weights(k)
    assert abs(w.sum() - 2.0) < 1e-14
    for m in range(2 * k):
        exact = 0.0 if m % 2 else 2.0 / (m + 1)
        assert abs(np.dot(w, x ** m) - exact) < 1e-13
    # not exact at degree 2k (GLL loses one degree against Gauss)
    assert abs(np.dot(w, x ** (2 * k)) - 2.0 / (2 * k + 1)) > 1e-6


@pytest.mark.parametrize("k", range(1, 9))
def test_derivative_matrix_exact_on_polynomials(k):
    x, _ = gll_nodes_weights(k)
    D = lagrange_derivative_matrix(x)
    np.testing.assert_allclose(D @ np.ones_like(x), 0.0, atol=1e-12)
    for m in range(1, k + 1):
        np.testing.assert_allclose(D @ x ** m, m * x ** (m - 1), atol=1e-11)


@pytest.mark.parametrize("k", [2, 3, 4])
def test_derivative_matrix_against_product_form(k):
    """D[i, j] = l_j'(x_i) with l_j built independently as a numpy Polynomial."""
    x, _ = gll_nodes_weights(k)
    D = lagrange_derivative_matrix(x)
    for j in range(k + 1):
        others = np.delete(x, j)
        lj = Polynomial.fromroots(others) / np.prod(x[j] - others)
        np.testing.assert_allclose(lj(x), np.eye(k + 1)[j], atol=1e-13)
        np.testing.assert_allclose(lj.deriv()(x), D[:, j], atol=1e-12)
        np.testing.assert_allclose(lagrange_eval(x, j, x), np.eye(k + 1)[j], atol=1e-14)


def test_minimum_spacings():
    """Smallest node gaps: 1.0 (k=2), 1 - 1/sqrt(5) (k=3), 1 - sqrt(3/7) (k=4)."""
    for k, gap in [(2, 1.0), (3, 1 - 1 / math.sqrt(5)), (4, 1 - math.sqrt(3 / 7))]:
        x, _ = gll_nodes_weights(k)
        assert abs(np.diff(x).min() - gap) < 1e-14
