"""Mesh side of the oracle: classification, ghost faces, active-DoF numbering.

Sec. 2: a Cartesian mesh of squares/cubes of size h; a level set phi, positive
inside the domain; cells are inside, cut or outside, and a cell takes part in
the computation when it meets the domain (Algorithm 1 loops over K with
K intersect Omega non-empty).  Sec. 2.2 and the figure of intersected cells:
the ghost penalty acts on faces between a cut cell and a cut or interior cell.

Readings taken where the paper is silent:
  * ball(s): exact interval test on each cell box.  With d_min / d_max the
    nearest / farthest distance from the centre to the box, the cell is
    inside if d_max^2 < r^2, outside if d_min^2 >= r^2 (a point with phi <= 0
    counts as outside), cut otherwise.  A union of balls is inside if one
    ball holds the whole cell, outside if every ball misses it, else cut.
  * gyroid and other smooth level sets: phi sampled on an (m+1)^d lattice per
    cell (m = 4), with the Lipschitz margin L * (h/m) * sqrt(d)/2 (L = sqrt 6
    for the gyroid): inside if min > margin, outside if max < -margin, else cut.
  * ghost face: interior face of the mesh between two active cells with at
    least one of them cut (``all_faces``: every interior face between active
    cells, used by the tests on full boxes).

Array conventions: cell arrays are indexed [ix, iy(, iz)]; lattice node arrays
[X, Y(, Z)] with X = ix*k + p.  The compact numbering orders active lattice
nodes lexicographically with x fastest (Sec. 2.4, i = i1 + i2 N1 + i3 N1 N2).
"""
from __future__ import annotations

import math

import numpy as np

from .basis import gauss_lobatto_nodes

OUTSIDE, CUT, INSIDE = 0, 1, 2
SAMPLES_PER_CELL = 4


def _cell_edges(pr, d):
    n = pr.n
    h = (pr.hi - pr.lo) / n
    i = np.arange(n, dtype=np.float64)
    lo = pr.lo + i * h
    hi = pr.lo + (i + 1.0) * h
    return lo, hi


def classify_cells(pr) -> np.ndarray:
    """int8 array (n,)*dim with OUTSIDE / CUT / INSIDE per cell."""
    d, n = pr.dim, pr.n
    shape = (n,) * d
    if pr.ls_kind == 4:  # constant level set
        v = INSIDE if pr.ls_value > 0 else OUTSIDE
        return np.full(shape, v, dtype=np.int8)
    if pr.ls_kind == 1:
        return _classify_balls(pr)
    if pr.ls_kind == 2:
        return _classify_sampled(pr)
    raise ValueError("unknown level-set kind")


def _classify_balls(pr) -> np.ndarray:
    d, n = pr.dim, pr.n
    lo, hi = _cell_edges(pr, d)
    any_inside = np.zeros((n,) * d, dtype=bool)
    all_outside = np.ones((n,) * d, dtype=bool)
    for c, r in zip(pr.centers, pr.radii):
        dmin2 = None
        dmax2 = None
        for a in range(d):
            near = np.maximum(np.maximum(lo - c[a], c[a] - hi), 0.0)
            far = np.maximum(np.abs(lo - c[a]), np.abs(hi - c[a]))
            shp = [1] * d
            shp[a] = n
            n2 = (near * near).reshape(shp)
            f2 = (far * far).reshape(shp)
            dmin2 = n2 if dmin2 is None else dmin2 + n2
            dmax2 = f2 if dmax2 is None else dmax2 + f2
        r2 = r * r
        any_inside |= np.broadcast_to(dmax2 < r2, (n,) * d)
        all_outside &= np.broadcast_to(dmin2 >= r2, (n,) * d)
    out = np.full((n,) * d, CUT, dtype=np.int8)
    out[all_outside] = OUTSIDE
    out[any_inside] = INSIDE
    return out


def _gyroid(x, y, z, iso):
    return ((np.sin(x) * np.cos(y) + np.sin(y) * np.cos(z)) + np.sin(z) * np.cos(x)) - iso


def _classify_sampled(pr) -> np.ndarray:
    d, n, m = pr.dim, pr.n, SAMPLES_PER_CELL
    assert d == 3
    hs = (pr.hi - pr.lo) / (n * m)
    coords = pr.lo + np.arange(n * m + 1, dtype=np.float64) * hs
    lip = math.sqrt(6.0)
    margin = lip * hs * math.sqrt(3.0) / 2.0
    cmin = np.full((n, n, n), np.inf)
    cmax = np.full((n, n, n), -np.inf)
    # sweep z planes of samples to bound memory
    X, Y = np.meshgrid(coords, coords, indexing="ij")
    for zs in range(n * m + 1):
        ph = _gyroid(X, Y, coords[zs], pr.iso)          # (nm+1, nm+1)
        # per cell (ix, iy): min/max over its (m+1)^2 samples in this plane
        win_min = np.full((n, n), np.inf)
        win_max = np.full((n, n), -np.inf)
        for p in range(m + 1):
            for q in range(m + 1):
                blk = ph[p:p + n * m:m, q:q + n * m:m]
                win_min = np.minimum(win_min, blk)
                win_max = np.maximum(win_max, blk)
        for iz in {zs // m, zs // m - 1} if zs % m == 0 else {zs // m}:
            if 0 <= iz < n:
                cmin[:, :, iz] = np.minimum(cmin[:, :, iz], win_min)
                cmax[:, :, iz] = np.maximum(cmax[:, :, iz], win_max)
    out = np.full((n, n, n), CUT, dtype=np.int8)
    out[cmax < -margin] = OUTSIDE
    out[cmin > margin] = INSIDE
    return out


def ghost_faces(pr, cls: np.ndarray):
    """Penalised faces as a list (one int64 array of lower cells per axis).

    Each entry is the multi-index array (nf_a, dim) of the lower cell K- of a
    face with normal along axis a; K+ = K- + e_a.  Sorted by the lexicographic
    (x fastest) index of K-.
    """
    d = pr.dim
    active = cls != OUTSIDE
    cut = cls == CUT
    out = []
    for a in range(d):
        sl_lo = [slice(None)] * d
        sl_hi = [slice(None)] * d
        sl_lo[a] = slice(0, pr.n - 1)
        sl_hi[a] = slice(1, pr.n)
        both = active[tuple(sl_lo)] & active[tuple(sl_hi)]
        if pr.all_faces:
            sel = both
        else:
            sel = both & (cut[tuple(sl_lo)] | cut[tuple(sl_hi)])
        idx = np.argwhere(sel)                       # C order: last axis fastest
        lin = _lex_index(idx, pr.n)
        order = np.argsort(lin, kind="stable")
        out.append(idx[order].astype(np.int64))
    return out


def _lex_index(mi: np.ndarray, n: int) -> np.ndarray:
    """Lexicographic index with the first coordinate fastest."""
    lin = np.zeros(mi.shape[0], dtype=np.int64)
    for a in reversed(range(mi.shape[1])):
        lin = lin * n + mi[:, a]
    return lin


class Numbering:
    """Active lattice nodes, numbered lexicographically with x fastest."""

    def __init__(self, pr, cls: np.ndarray):
        d, n, k = pr.dim, pr.n, pr.degree
        self.dim, self.n, self.k = d, n, k
        nl = n * k + 1
        active = cls != OUTSIDE
        node = np.zeros((nl,) * d, dtype=bool)
        # a lattice node is active when it is a node of an active cell
        for off in np.ndindex(*((k + 1,) * d)):
            sl = tuple(slice(o, o + k * (n - 1) + 1, k) for o in off)
            node[sl] |= active
        flat = node.ravel(order="F")
        num = np.cumsum(flat, dtype=np.int64) - 1
        cmap = np.where(flat, num, -1)
        self.n_active = int(flat.sum())
        self.cmap = cmap.reshape(node.shape, order="F")
        self.node = node
        self.xi = gauss_lobatto_nodes(k)
        self.lo, self.h = pr.lo, (pr.hi - pr.lo) / n

    def lattice_coord(self, X: np.ndarray) -> np.ndarray:
        """Physical coordinate of lattice index X along one axis (GL nodes inside each cell)."""
        X = np.asarray(X)
        ci = X // self.k
        p = X % self.k
        return self.lo + (ci + self.xi[p]) * self.h

    def coords(self) -> np.ndarray:
        """(n_active, dim) physical coordinates of the active DoFs in compact order."""
        idx = np.argwhere(self.node.transpose())[:, ::-1]  # x fastest ordering
        return np.stack([self.lattice_coord(idx[:, a]) for a in range(self.dim)], axis=1)

    def patch_index(self, axis: int, lower: np.ndarray) -> np.ndarray:
        """(nf, P) compact indices of the two-cell patch of each face.

        Patch-local order is lexicographic over the patch box with x fastest;
        the box has 2k+1 nodes along ``axis`` and k+1 along the others (Sec. 2.4:
        N_1 = 2k+1 for the normal direction, N_i = k+1 otherwise).
        """
        d, k = self.dim, self.k
        ext = [2 * k + 1 if a == axis else k + 1 for a in range(d)]
        loc = np.array(list(np.ndindex(*ext[::-1])))[:, ::-1]   # x fastest
        base = lower * k                                          # (nf, d)
        lat = base[:, None, :] + loc[None, :, :]                  # (nf, P, d)
        out = self.cmap[tuple(lat[..., a] for a in range(d))]
        if np.any(out < 0):
            raise AssertionError("patch touches an inactive node")
        return out
