"""Slab partitions of the active mesh for distributed evaluation (int64 / float64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

What the paper fixes (Sec. 2.7, and the two communication steps of Algorithm 1):
  * every cell gets a weight: 0 outside the domain, 1 strictly inside, k^(d-1)
    for a cut cell, and the cells are distributed so that the weight sums of the
    ranks are balanced;
  * a face shared by two ranks is evaluated by the one with the lower rank;
  * the values of u on ghost entries are imported before the face loop, and the
    contributions to ghost entries of w are sent to their owners and added there.

Readings (the paper names no partitioner; deal.II's is not described):
  * a partition is a slab of whole cell layers [b_p, b_{p+1}) along the last
    axis (y in 2D, z in 3D), the slowest index of the numbering;
  * b_p is the first layer boundary l with C_l * P >= p * C_n, where C_l is the
    weight of layers 0..l-1 and P the number of partitions; then b_p is clamped
    to [2p, n - 2(P - p)] and raised to b_{p-1} + 2, so that every slab has at
    least two layers;
  * a lattice node on plane Z of the last axis belongs to the partition p with
    b_p k <= Z < b_{p+1} k (the last partition also owns Z = n k);
  * rank r keeps the active DoFs on planes [b_r k, min(b_{r+1} + 1, n) k]: its own
    planes plus one cell of halo above (the faces it owns reach no lower plane).
"""
from __future__ import annotations

import numpy as np

from . import mesh as omesh


def layer_weights(pr, cls: np.ndarray) -> np.ndarray:
    """Weight of each cell layer along the last axis (int64, length n)."""
    d, k = pr.dim, pr.degree
    w = np.where(cls == omesh.INSIDE, 1, np.where(cls == omesh.CUT, k ** (d - 1), 0)).astype(np.int64)
    # cls is indexed [ix, iy(, iz)]: sum over every axis but the last
    return w.sum(axis=tuple(range(d - 1)))


def slab_bounds(pr, nparts: int, cls: np.ndarray | None = None) -> np.ndarray:
    """Layer boundaries 0 = b_0 < ... < b_P = n (int64, length nparts + 1)."""
    n = pr.n
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    if nparts > 1 and n < 2 * nparts:
        raise ValueError("fewer than two cell layers per partition")
    if cls is None:
        cls = omesh.classify_cells(pr)
    C = np.concatenate([[0], np.cumsum(layer_weights(pr, cls))])
    b = np.zeros(nparts + 1, dtype=np.int64)
    b[nparts] = n
    for p in range(1, nparts):
        reach = np.nonzero(C * nparts >= p * C[-1])[0]
        q = int(reach[0]) if reach.size else n
        q = max(q, 2 * p)
        q = min(q, n - 2 * (nparts - p))
        q = max(q, int(b[p - 1]) + 2)
        b[p] = q
    return b


def cell_rank(bounds: np.ndarray, layer: np.ndarray) -> np.ndarray:
    """Partition holding the cells of the given layers."""
    return np.searchsorted(bounds, layer, side="right") - 1


def face_owner(pr, faces, bounds: np.ndarray):
    """Per axis: the rank that evaluates each face, the lower of its two cells' ranks."""
    out = []
    for a, lower in enumerate(faces):
        upper = lower.copy()
        upper[:, a] += 1
        r0 = cell_rank(bounds, lower[:, -1])
        r1 = cell_rank(bounds, upper[:, -1])
        out.append(np.minimum(r0, r1))
    return out


def plane_of_dofs(num: omesh.Numbering) -> np.ndarray:
    """Lattice coordinate along the last axis of every active DoF, in compact order."""
    idx = np.argwhere(num.node.transpose())   # last axis first: compact order
    return idx[:, 0].astype(np.int64)


def window(pr, num: omesh.Numbering, bounds: np.ndarray, r: int) -> dict:
    """offset / n_local / n_owned / n_lower of partition r (compact numbering)."""
    k, n = pr.degree, pr.n
    Z = plane_of_dofs(num)
    lo, hi = int(bounds[r]), int(bounds[r + 1])
    top = min(hi + 1, n) * k
    n_local = int(np.count_nonzero((Z >= lo * k) & (Z <= top)))
    offset = int(np.count_nonzero(Z < lo * k))
    own_top = hi * k if hi < n else n * k + 1
    n_owned = int(np.count_nonzero((Z >= lo * k) & (Z < own_top)))
    n_lower = int(np.count_nonzero((Z >= lo * k) & (Z <= (lo + 1) * k))) if lo > 0 else 0
    return {"layer_lo": lo, "layer_hi": hi, "offset": offset, "n_local": n_local,
            "n_owned": n_owned, "n_lower": n_lower, "n_global": int(num.n_active)}
