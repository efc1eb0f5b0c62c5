"""Explicit face matrices and y = G x (float64, numpy).

Definition followed (Sec. 2.2, g_F; Sec. 2.4, entries of the face matrix):

    A_F[I, J] = sum_{j=1..k} c_j h^{2j-1} integral_F [d_n^j phi_J] [d_n^j phi_I] ds

for the patch DoFs I, J of the two cells K-, K+ sharing F.  [v] = v|K- - v|K+.
phi_I restricted to a cell is the tensor product of 1D Lagrange polynomials
on that cell's Gauss-Lobatto points (Eq. of the tensor-product basis), or 0
when node I is not a node of the cell.  The normal derivative of order j of
the restriction is taken in physical coordinates at the face; the face
integral uses a tensor Gauss-Legendre rule with k+1 points per tangential
direction (exact: the integrand has degree 2k in each tangential variable).

Readings (the paper is ambiguous or silent here):
  * sum over j = 1..k (the j = 0 jump vanishes for continuous FE_Q);
  * gamma enters once, through the per-order weights c_j (default c_j = gamma,
    option c_j = gamma / (j!)^2 as in the g_F formula);
  * h is the cell edge length (the g_F text says "diameter of the face").
"""
from __future__ import annotations

import numpy as np

from . import mesh as omesh
from .basis import gauss_legendre, gauss_lobatto_nodes, lagrange_derivative_at, lagrange_value


def face_matrix(dim: int, k: int, h: float, axis: int, cweights, origin=None) -> np.ndarray:
    """Dense (P x P) face matrix of one face with normal along ``axis``.

    ``origin`` is the physical position of the face's lowest corner (the face
    lies in the plane x_axis = origin[axis]); it defaults to 0.  The patch
    ordering is lexicographic with x fastest over a box of 2k+1 nodes along
    the normal and k+1 along each tangential direction.
    """
    cweights = np.asarray(cweights, dtype=np.float64)
    assert cweights.shape == (k,)
    if origin is None:
        origin = np.zeros(dim)
    origin = np.asarray(origin, dtype=np.float64)
    xi = gauss_lobatto_nodes(k)
    xf = origin[axis]
    nodes_lo = xf - h + h * xi          # K- along the normal
    nodes_hi = xf + h * xi              # K+ along the normal
    tang = [a for a in range(dim) if a != axis]
    tnodes = {a: origin[a] + h * xi for a in tang}
    tq = {a: gauss_legendre(k + 1, origin[a], origin[a] + h) for a in tang}

    ext = [2 * k + 1 if a == axis else k + 1 for a in range(dim)]
    loc = np.array(list(np.ndindex(*ext[::-1])))[:, ::-1]      # (P, dim), x fastest
    P = loc.shape[0]

    # tensor quadrature on the face
    qpts = [tq[a][0] for a in tang]
    qwts = [tq[a][1] for a in tang]
    grids = np.meshgrid(*qpts, indexing="ij")
    wgrid = np.ones_like(grids[0])
    for g, w in zip(range(len(tang)), qwts):
        shp = [1] * len(tang)
        shp[g] = len(w)
        wgrid = wgrid * w.reshape(shp)
    W = wgrid.ravel()
    Q = W.size
    qcoord = {a: grids[t].ravel() for t, a in enumerate(tang)}

    # jumps [d_n^j phi_I](x_q): shape (k, Q, P)
    jump = np.zeros((k, Q, P))
    for I in range(P):
        b = loc[I, axis]
        tval = np.ones(Q)
        for a in tang:
            tval = tval * lagrange_value(tnodes[a], int(loc[I, a]), qcoord[a])
        for j in range(1, k + 1):
            dlo = lagrange_derivative_at(nodes_lo, b, xf, j) if b <= k else 0.0
            dhi = lagrange_derivative_at(nodes_hi, b - k, xf, j) if b >= k else 0.0
            jump[j - 1, :, I] = (dlo - dhi) * tval

    A = np.zeros((P, P))
    for j in range(1, k + 1):
        Jj = jump[j - 1]
        A += cweights[j - 1] * h ** (2 * j - 1) * (Jj.T * W) @ Jj
    return A


class Oracle:
    """Everything the oracle needs for one problem (a workloads.Problem)."""

    def __init__(self, pr, number: bool = True):
        self.pr = pr
        self.cls = omesh.classify_cells(pr)
        self.faces = omesh.ghost_faces(pr, self.cls)
        self.num = omesh.Numbering(pr, self.cls) if number else None
        self._A = {}
        self._pidx = {}

    @property
    def n_active(self) -> int:
        return self.num.n_active

    @property
    def n_faces(self) -> int:
        return int(sum(f.shape[0] for f in self.faces))

    def A(self, axis: int) -> np.ndarray:
        """One explicit face matrix per axis: on a uniform Cartesian mesh every
        face of a given normal direction has the same matrix (Sec. 2.2).  For a
        problem with the macro-patch stabilisation, its matrix (oracle.macro_patch)."""
        if axis not in self._A:
            pr = self.pr
            if getattr(pr, "stabilization", 0) == 1:
                from .macro_patch import face_matrix_macro
                self._A[axis] = face_matrix_macro(pr.dim, pr.degree, pr.h, axis, pr.gamma)
            else:
                self._A[axis] = face_matrix(pr.dim, pr.degree, pr.h, axis, pr.cweights())
        return self._A[axis]

    def patch_index(self, axis: int) -> np.ndarray:
        if axis not in self._pidx:
            self._pidx[axis] = self.num.patch_index(axis, self.faces[axis])
        return self._pidx[axis]

    def apply(self, x: np.ndarray, face_mask=None) -> np.ndarray:
        """y = G x: loop over faces, y[patch] += A_F x[patch] (Algorithm 1, face loop).

        ``face_mask`` (one bool array per axis) restricts the loop to a subset of
        the faces, e.g. those one rank evaluates (Sec. 2.7).
        """
        x = np.asarray(x, dtype=np.float64)
        y = np.zeros(self.n_active)
        for a in range(self.pr.dim):
            idx = self.patch_index(a)
            if face_mask is not None:
                idx = idx[face_mask[a]]
            if idx.shape[0] == 0:
                continue
            yf = x[idx] @ self.A(a).T
            y += np.bincount(idx.ravel(), weights=yf.ravel(), minlength=self.n_active)
        return y

    def apply_rows(self, x: np.ndarray, rows: np.ndarray) -> np.ndarray:
        """(G x)[rows], using only the faces whose patch contains one of ``rows``."""
        x = np.asarray(x, dtype=np.float64)
        rows = np.asarray(rows, dtype=np.int64)
        y = np.zeros(self.n_active)
        want = np.zeros(self.n_active, dtype=bool)
        want[rows] = True
        for a in range(self.pr.dim):
            idx = self.patch_index(a)
            if idx.shape[0] == 0:
                continue
            hit = want[idx].any(axis=1)
            sub = idx[hit]
            yf = x[sub] @ self.A(a).T
            y += np.bincount(sub.ravel(), weights=yf.ravel(), minlength=self.n_active)
        return y[rows]

    def energy(self, x: np.ndarray) -> float:
        """x^T G x = sum_F x_F^T A_F x_F."""
        e = 0.0
        for a in range(self.pr.dim):
            idx = self.patch_index(a)
            if idx.shape[0] == 0:
                continue
            xf = x[idx]
            e += float(np.einsum("fi,ij,fj->", xf, self.A(a), xf))
        return e

    def face_list(self):
        """(axis, lower-cell lexicographic index) of every face, in output order."""
        out = []
        n = self.pr.n
        for a, f in enumerate(self.faces):
            lin = np.zeros(f.shape[0], dtype=np.int64)
            for ax in reversed(range(self.pr.dim)):
                lin = lin * n + f[:, ax]
            out.append(np.stack([np.full(f.shape[0], a, dtype=np.int64), lin], axis=1))
        return np.concatenate(out) if out else np.zeros((0, 2), dtype=np.int64)
