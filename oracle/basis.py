"""1D ingredients of the oracle (float64, numpy).

Sec. 2.4 builds every shape function as a product of 1D Lagrange polynomials
phi_i(x_1) phi_i(x_2) phi_i(x_3).  The elements are FE_Q of degree k with
Gauss-Lobatto support points.  Derivatives of order j of a 1D Lagrange
polynomial are read off its expansion in powers of (x - x0): the j-th
derivative at x0 is j! times the j-th coefficient.  The expansion multiplies
the linear factors (x - x_i)/(x_m - x_i) one by one, so no differentiation
matrix is involved.
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import legendre as npleg


def gauss_lobatto_nodes(k: int) -> np.ndarray:
    """k+1 Gauss-Lobatto points on [0, 1]: the end points and the roots of P_k'.

    Element support points of FE_Q(k) (Sec. 2, Lagrange elements of order k).
    """
    if k < 1:
        raise ValueError("degree must be >= 1")
    if k == 1:
        return np.array([0.0, 1.0])
    c = np.zeros(k + 1)
    c[k] = 1.0
    dc = npleg.legder(c)            # P_k' in the Legendre basis
    ddc = npleg.legder(dc)
    r = np.sort(npleg.legroots(dc).real)
    for _ in range(4):              # Newton polish of the companion-matrix roots
        r = r - npleg.legval(r, dc) / npleg.legval(r, ddc)
    t = np.concatenate(([-1.0], r, [1.0]))
    return 0.5 * (t + 1.0)


def gauss_legendre(nq: int, a: float, b: float):
    """Gauss-Legendre rule with nq points on [a, b] (exact to degree 2 nq - 1)."""
    t, w = npleg.leggauss(nq)
    return a + 0.5 * (b - a) * (t + 1.0), 0.5 * (b - a) * w


def lagrange_taylor(nodes: np.ndarray, m: int, x0: float) -> np.ndarray:
    """Coefficients a_p, p = 0..len(nodes)-1, with l_m(x) = sum_p a_p (x - x0)^p.

    l_m is the Lagrange polynomial that is 1 at nodes[m] and 0 at the other nodes.
    Each factor (x - x_i)/(x_m - x_i) is written as ((x - x0) + (x0 - x_i))/(x_m - x_i)
    and multiplied in with a polynomial convolution.
    """
    coef = np.array([1.0])
    for i, xi in enumerate(nodes):
        if i == m:
            continue
        lin = np.array([x0 - xi, 1.0]) / (nodes[m] - xi)
        coef = np.convolve(coef, lin)
    return coef


def lagrange_derivative_at(nodes: np.ndarray, m: int, x0: float, j: int) -> float:
    """d^j/dx^j l_m at x0 = j! * (coefficient of (x - x0)^j)."""
    coef = lagrange_taylor(nodes, m, x0)
    if j >= len(coef):
        return 0.0
    return math.factorial(j) * coef[j]


def lagrange_value(nodes: np.ndarray, m: int, x) -> np.ndarray:
    """l_m(x) by the product formula."""
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    for i, xi in enumerate(nodes):
        if i == m:
            continue
        out = out * (x - xi) / (nodes[m] - xi)
    return out
