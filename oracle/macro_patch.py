"""Macro-patch stabilisation: the explicit face matrix (float64, numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2.2 names, next to the ghost penalty, the macro-patch stabilisation: the
difference between a function on an element and the extension of the function
from the neighbouring element, squared and integrated.  Reading (the paper gives
no formula): per ghost face F with cells K-, K+,

    s_F(u, v) = gamma * sum_{K in {K-, K+}} integral_K (u|_K - E_K' u|_K') (v|_K - E_K' v|_K') dx

with K' the other cell and E_K' u|_K' the polynomial of u on K' evaluated in K
(its extension).  The oracle evaluates this by d-dimensional Gauss quadrature
(k+1 points per direction in each cell, exact for the degree-2k integrands) of
the tensor Lagrange basis of each cell, evaluated inside and outside that cell,
and assembles the dense P x P matrix; it uses no factorisation.
"""
from __future__ import annotations

import numpy as np

from .basis import gauss_legendre, gauss_lobatto_nodes, lagrange_value


def face_matrix_macro(dim: int, k: int, h: float, axis: int, gamma: float, origin=None) -> np.ndarray:
    """Dense (P x P) macro-patch matrix of one face with normal along ``axis`` (patch order
    lexicographic, x fastest, 2k+1 nodes along the normal and k+1 along the others)."""
    if origin is None:
        origin = np.zeros(dim)
    origin = np.asarray(origin, dtype=np.float64)
    xi = gauss_lobatto_nodes(k)
    xf = origin[axis]
    ext = [2 * k + 1 if a == axis else k + 1 for a in range(dim)]
    loc = np.array(list(np.ndindex(*ext[::-1])))[:, ::-1]      # (P, dim), x fastest
    P = loc.shape[0]
    # nodes of each cell along each axis; cell c = 0 is K-, 1 is K+
    def cell_nodes(c, a):
        if a == axis:
            return xf - h + c * h + h * xi
        return origin[a] + h * xi
    def cell_lo(c, a):
        return xf - h + c * h if a == axis else origin[a]
    A = np.zeros((P, P))
    for c in (0, 1):
        other = 1 - c
        # Gauss points of cell c
        qp = [gauss_legendre(k + 1, cell_lo(c, a), cell_lo(c, a) + h) for a in range(dim)]
        grids = np.meshgrid(*[q[0] for q in qp], indexing="ij")
        wg = np.ones_like(grids[0])
        for a in range(dim):
            shp = [1] * dim
            shp[a] = k + 1
            wg = wg * qp[a][1].reshape(shp)
        W = wg.ravel()
        X = [g.ravel() for g in grids]
        # value at the points of the polynomial of phi_I on cell cc (0 if I is not a node of cc)
        def values(cc):
            V = np.zeros((W.size, P))
            for I in range(P):
                b = int(loc[I, axis])
                lb = b - k * cc                      # index along the normal within cell cc
                if lb < 0 or lb > k:
                    continue
                v = np.ones(W.size)
                for a in range(dim):
                    m = lb if a == axis else int(loc[I, a])
                    v = v * lagrange_value(cell_nodes(cc, a), m, X[a])
                V[:, I] = v
            return V
        D = values(c) - values(other)
        A += gamma * (D.T * W) @ D
    return A
