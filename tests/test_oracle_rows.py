"""Pin of the oracle's sampled apply, Oracle.apply_rows.

The sampled GPU parity tests on the large meshes compare against
apply_rows(x, rows), which evaluates only the faces whose patch holds one of
``rows``.  It must give exactly (G x)[rows] of the full face loop (Algorithm 1):
a face left out by the patch test, or a row summed twice, changes the value by
the size of a face contribution.  Checked against the full apply on 2D and 3D
meshes, with random rows, rows on the patches of single faces, every row, no
row, and rows that no face touches.
"""
import numpy as np
import pytest

from oracle.ghost_penalty import Oracle
from paper_2503_00246_gb300 import workloads as W


def _cases():
    return [W.small_ball(2, 14, 3, seed=41), W.small_ball(3, 8, 2, seed=42),
            W.small_ball(3, 7, 4, seed=43, weights=W.paper_weights(0.5, 4))]


@pytest.mark.parametrize("case", range(3))
def test_apply_rows_equals_full_apply(case):
    pr = _cases()[case]
    o = Oracle(pr)
    x = W.x_vectors(pr, o.n_active)[0]
    full = o.apply(x)
    scale = np.abs(full).max()
    rng = np.random.default_rng(5 + case)
    patch_rows = np.unique(np.concatenate([o.patch_index(a)[rng.integers(0, o.faces[a].shape[0], 3)].ravel()
                                           for a in range(pr.dim) if o.faces[a].shape[0] > 0]))
    untouched = np.flatnonzero(full == 0.0)
    sets = {"random": np.unique(rng.integers(0, o.n_active, 200)), "patches": patch_rows,
            "all": np.arange(o.n_active), "none": np.zeros(0, dtype=np.int64),
            "untouched": untouched[:50]}
    for name, rows in sets.items():
        got = o.apply_rows(x, rows)
        assert got.shape == rows.shape, name
        # the same faces summed in the same order; only the matrix products' blocking may differ
        assert np.abs(got - full[rows]).max(initial=0.0) <= 1e-14 * scale, name
    assert untouched.size > 0 and np.all(o.apply_rows(x, untouched[:50]) == 0.0)


def test_apply_rows_sees_every_face_of_a_row():
    """A row on a cell corner receives contributions from several faces of every axis;
    dropping any one face of its patch set changes the result."""
    pr = W.box_problem(3, 4, 2, all_faces=True)
    o = Oracle(pr)
    x = W.x_vectors(pr, o.n_active)[0]
    xyz = o.num.coords()
    h = pr.h
    mid = np.flatnonzero(np.all(np.isclose(xyz, pr.lo + 2 * h), axis=1))   # the central lattice node
    assert mid.size == 1
    got = o.apply_rows(x, mid)[0]
    assert abs(got - o.apply(x)[mid[0]]) <= 1e-14 * np.abs(o.apply(x)).max()
    # the same node without the faces of one axis differs by that axis' share
    masks = [np.ones(o.faces[a].shape[0], dtype=bool) for a in range(3)]
    masks[1][:] = False
    assert abs(o.apply(x, face_mask=masks)[mid[0]] - got) > 1e-6 * abs(got)
