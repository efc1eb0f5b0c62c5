"""Pins of the oracle's 1D pieces against closed forms and reproduction identities."""
import math

import numpy as np
import pytest

from oracle.basis import (gauss_legendre, gauss_lobatto_nodes, lagrange_derivative_at,
                          lagrange_taylor, lagrange_value)


def test_gauss_lobatto_closed_forms():
    # interior GL points on [0,1]: k=2 midpoint; k=3 (1 -+ 1/sqrt5)/2; k=4 1/2, (1 -+ sqrt(3/7))/2
    np.testing.assert_allclose(gauss_lobatto_nodes(1), [0.0, 1.0], atol=0)
    np.testing.assert_allclose(gauss_lobatto_nodes(2), [0.0, 0.5, 1.0], atol=1e-15)
    s5 = 1.0 / math.sqrt(5.0)
    np.testing.assert_allclose(gauss_lobatto_nodes(3), [0.0, (1 - s5) / 2, (1 + s5) / 2, 1.0],
                               atol=1e-15)
    s = math.sqrt(3.0 / 7.0)
    np.testing.assert_allclose(gauss_lobatto_nodes(4), [0.0, (1 - s) / 2, 0.5, (1 + s) / 2, 1.0],
                               atol=1e-15)


@pytest.mark.parametrize("k", range(1, 11))
def test_gauss_lobatto_symmetric_and_quadrature_exact(k):
    x = gauss_lobatto_nodes(k)
    assert x[0] == 0.0 and x[-1] == 1.0
    np.testing.assert_allclose(x + x[::-1], 1.0, atol=1e-15)
    assert np.all(np.diff(x) > 0)
    # GL rule with these nodes integrates degree 2k-1 exactly: weights = int of Lagrange basis
    if k >= 2:
        xg, wg = gauss_legendre(k + 1, 0.0, 1.0)
        w = np.array([np.dot(wg, lagrange_value(x, m, xg)) for m in range(k + 1)])
        for p in range(2 * k):
            np.testing.assert_allclose(np.dot(w, x ** p), 1.0 / (p + 1), rtol=1e-13)


@pytest.mark.parametrize("nq", [1, 2, 3, 5, 9])
def test_gauss_legendre_exact(nq):
    a, b = -0.3, 1.7
    x, w = gauss_legendre(nq, a, b)
    for p in range(2 * nq):
        exact = (b ** (p + 1) - a ** (p + 1)) / (p + 1)
        np.testing.assert_allclose(np.dot(w, x ** p), exact, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_lagrange_cardinal_property(k):
    nodes = 0.3 + 0.7 * gauss_lobatto_nodes(k)
    for m in range(k + 1):
        for i, xi in enumerate(nodes):
            # Taylor form about another point, evaluated at the node
            c = lagrange_taylor(nodes, m, 0.11)
            terms = np.array([cp * (xi - 0.11) ** p for p, cp in enumerate(c)])
            assert abs(terms.sum() - (1.0 if i == m else 0.0)) <= 1e-14 * np.abs(terms).sum()


@pytest.mark.parametrize("k", [1, 2, 3, 4, 6, 8])
def test_lagrange_derivatives_reproduce_monomials(k):
    # sum_m x_m^p l_m(x) = x^p for p <= k, so the j-th derivatives at x0 satisfy
    # sum_m x_m^p l_m^(j)(x0) = p!/(p-j)! x0^(p-j).
    nodes = -0.4 + 0.9 * gauss_lobatto_nodes(k)
    x0 = nodes[-1]
    for j in range(0, k + 2):
        d = np.array([lagrange_derivative_at(nodes, m, x0, j) for m in range(k + 1)])
        for p in range(k + 1):
            lhs = np.dot(nodes ** p, d)
            rhs = 0.0 if j > p else math.factorial(p) / math.factorial(p - j) * x0 ** (p - j)
            scale = np.abs(nodes ** p * d).sum() + abs(rhs)
            assert abs(lhs - rhs) <= 1e-12 * scale + 1e-14
