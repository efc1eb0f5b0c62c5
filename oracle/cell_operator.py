"""Mass + Laplace stiffness over the active cells, and the model SPD system (float64).

The model system of the defect-correction study is (M_active + K_active + G) u = b:
the mass and stiffness of every active cell integrated over the whole cell (no cut
quadrature), plus the ghost penalty G.  Interior cells of the paper are treated
this way (Sec. 2.5.2: gradients at the k+1 Gauss points per direction, weighted
by the Jacobian and the quadrature weight, integrated against the test gradients).

The oracle builds one explicit ((k+1)^d x (k+1)^d) cell matrix by d-dimensional
Gauss quadrature of products of the tensor Lagrange basis and its gradient in
physical coordinates (k+2 points per direction, exact for the degree-2k
integrands), then assembles y = sum_K E_K^T (M_K + K_K) E_K x over the active cells.
No Kronecker factorisation is used.
"""
from __future__ import annotations

import numpy as np

from . import mesh as omesh
from .basis import gauss_legendre, gauss_lobatto_nodes, lagrange_derivative_at, lagrange_value


def cell_matrices(dim: int, k: int, h: float):
    """(M_K, K_K) of one cell [0,h]^dim, lexicographic node order with x fastest."""
    xi = h * gauss_lobatto_nodes(k)
    xq, wq = gauss_legendre(k + 2, 0.0, h)
    nq = xq.size
    # 1D values and first derivatives of the Lagrange basis at the Gauss points
    val = np.array([[lagrange_value(xi, m, x) for x in xq] for m in range(k + 1)])          # (k+1, nq)
    der = np.array([[lagrange_derivative_at(xi, m, x, 1) for x in xq] for m in range(k + 1)])
    loc = np.array(list(np.ndindex(*([k + 1] * dim))))[:, ::-1]                              # x fastest
    qloc = np.array(list(np.ndindex(*([nq] * dim))))[:, ::-1]
    nb = loc.shape[0]
    phi = np.ones((nb, qloc.shape[0]))
    grad = np.ones((dim, nb, qloc.shape[0]))
    w = np.ones(qloc.shape[0])
    for a in range(dim):
        w = w * wq[qloc[:, a]]
    for I in range(nb):
        for a in range(dim):
            va = val[loc[I, a]][qloc[:, a]]
            phi[I] = phi[I] * va
            for g in range(dim):
                grad[g, I] = grad[g, I] * (der[loc[I, a]][qloc[:, a]] if g == a else va)
    M = (phi * w) @ phi.T
    K = sum((grad[g] * w) @ grad[g].T for g in range(dim))
    return M, K


class CellOperator:
    """y = (M_active + K_active) x with the oracle's numbering (see oracle.mesh.Numbering)."""

    def __init__(self, pr, num: omesh.Numbering, cls: np.ndarray):
        self.pr, self.num = pr, num
        d, k, n = pr.dim, pr.degree, pr.n
        self.M, self.K = cell_matrices(d, k, pr.h)
        act = np.argwhere(cls != omesh.OUTSIDE)                       # (ncell, d) multi-indices
        loc = np.array(list(np.ndindex(*([k + 1] * d))))[:, ::-1]
        lat = act[:, None, :] * k + loc[None, :, :]
        self.idx = num.cmap[tuple(lat[..., a] for a in range(d))]     # (ncell, (k+1)^d)
        assert np.all(self.idx >= 0)

    def apply(self, x: np.ndarray, mass: float = 1.0, stiff: float = 1.0) -> np.ndarray:
        A = mass * self.M + stiff * self.K
        yc = x[self.idx] @ A.T
        return np.bincount(self.idx.ravel(), weights=yc.ravel(), minlength=self.num.n_active)
