"""Pins of oracle.partition (Sec. 2.7: weighted load balance, lowest-rank face
ownership, ghost import / contribution export of Algorithm 1).

The checks use facts the partition rules fix without reusing their formulas:
closed-form bounds for a uniformly weighted box, the weight total from the
classification counts, the lowest-rank rule restated through cell ranks, the
DoF windows against a brute-force walk over lattice nodes, and the exchange
invariant: the per-rank face loops plus the two exchanges give G x exactly.
"""
import numpy as np
import pytest

import oracle.mesh as omesh
import oracle.partition as opart
from oracle.ghost_penalty import Oracle
from paper_2503_00246_gb300 import workloads as W


def _problems():
    return [W.small_ball(3, 12, 2, radius=0.6, seed=3), W.small_ball(2, 20, 3, radius=0.7, seed=4),
            W.small_ball(3, 10, 3, radius=0.8, seed=5)]


@pytest.mark.parametrize("n,P", [(8, 2), (12, 3), (13, 4), (40, 7), (9, 4)])
def test_uniform_box_bounds_closed_form(n, P):
    # every cell inside and weighted 1: b_p = ceil(p n / P)
    pr = W.box_problem(3, n, 2)
    b = opart.slab_bounds(pr, P)
    want = [0] + [-(-p * n // P) for p in range(1, P)] + [n]
    assert b.tolist() == want


def test_weight_total_and_layers():
    for pr in _problems():
        cls = omesh.classify_cells(pr)
        w = opart.layer_weights(pr, cls)
        assert w.shape == (pr.n,)
        n_in = int(np.count_nonzero(cls == omesh.INSIDE))
        n_cut = int(np.count_nonzero(cls == omesh.CUT))
        assert int(w.sum()) == n_in + pr.degree ** (pr.dim - 1) * n_cut
        # layer l holds exactly the cells whose last index is l
        for l in (0, pr.n // 2, pr.n - 1):
            layer = cls[..., l]
            assert w[l] == np.count_nonzero(layer == omesh.INSIDE) + \
                pr.degree ** (pr.dim - 1) * np.count_nonzero(layer == omesh.CUT)


@pytest.mark.parametrize("P", [1, 2, 3, 4])
def test_bounds_valid_and_balanced(P):
    for pr in _problems():
        if pr.n < 2 * P:
            continue
        cls = omesh.classify_cells(pr)
        b = opart.slab_bounds(pr, P, cls)
        assert b[0] == 0 and b[-1] == pr.n
        if P > 1:
            assert np.all(np.diff(b) >= 2)
        w = opart.layer_weights(pr, cls)
        tot = w.sum()
        # where the clamp did not act, the slab weights deviate from the ideal by
        # less than one layer's weight
        parts = np.array([w[b[p]:b[p + 1]].sum() for p in range(P)])
        assert parts.sum() == tot
        for p in range(1, P):
            C = w[:b[p]].sum()
            if 2 * p < b[p] < pr.n - 2 * (P - p) and b[p] > b[p - 1] + 2:
                assert C * P >= p * tot and (C - w[b[p] - 1]) * P < p * tot


def test_bounds_errors():
    with pytest.raises(ValueError):
        opart.slab_bounds(W.box_problem(3, 5, 1), 3)
    with pytest.raises(ValueError):
        opart.slab_bounds(W.box_problem(3, 5, 1), 0)


def test_face_owner_is_lowest_rank():
    for pr in _problems():
        o = Oracle(pr)
        b = opart.slab_bounds(pr, 3 if pr.n >= 6 else 2, o.cls)
        owners = opart.face_owner(pr, o.faces, b)
        # brute force: rank of every cell by walking the slabs, min over the two cells
        rank_of_layer = np.zeros(pr.n, dtype=np.int64)
        for p in range(len(b) - 1):
            for l in range(b[p], b[p + 1]):
                rank_of_layer[l] = p
        for a, lower in enumerate(o.faces):
            for i, cell in enumerate(lower):
                up = cell.copy()
                up[a] += 1
                assert owners[a][i] == min(rank_of_layer[cell[-1]], rank_of_layer[up[-1]])
                # the lower cell always has the lower rank: the owner is its slab
                assert owners[a][i] == rank_of_layer[cell[-1]]


def test_windows_brute_force():
    for pr in _problems():
        o = Oracle(pr)
        k, n, d = pr.degree, pr.n, pr.dim
        P = 3 if n >= 6 else 2
        b = opart.slab_bounds(pr, P, o.cls)
        # brute force: walk the lattice in compact order and record each node's plane
        planes = []
        for Z in range(n * k + 1):
            sl = [slice(None)] * d
            sl[-1] = Z
            planes += [Z] * int(np.count_nonzero(o.num.node[tuple(sl)]))
        planes = np.array(planes)
        assert planes.size == o.n_active
        tot_owned = 0
        for r in range(P):
            win = opart.window(pr, o.num, b, r)
            lo, hi = b[r] * k, min(b[r + 1] + 1, n) * k
            idx = np.nonzero((planes >= lo) & (planes <= hi))[0]
            assert win["offset"] == (idx[0] if idx.size else np.count_nonzero(planes < lo))
            assert win["n_local"] == idx.size
            assert np.all(np.diff(idx) == 1)                 # a contiguous block
            tot_owned += win["n_owned"]
            if r + 1 < P:
                nxt = opart.window(pr, o.num, b, r + 1)
                assert win["offset"] + win["n_owned"] == nxt["offset"]
                assert win["n_local"] - win["n_owned"] == nxt["n_lower"]
            else:
                assert win["n_owned"] == win["n_local"]
        assert tot_owned == o.n_active


def test_owned_patches_inside_window():
    for pr in _problems():
        o = Oracle(pr)
        P = 3 if pr.n >= 6 else 2
        b = opart.slab_bounds(pr, P, o.cls)
        owners = opart.face_owner(pr, o.faces, b)
        for r in range(P):
            win = opart.window(pr, o.num, b, r)
            for a in range(pr.dim):
                idx = o.patch_index(a)[owners[a] == r]
                if idx.size:
                    assert idx.min() >= win["offset"]
                    assert idx.max() < win["offset"] + win["n_local"]


def test_exchange_reproduces_global_apply():
    # Algorithm 1 with ranks: import the halo of x, loop over the own faces, add the
    # halo contributions to the rank above.  The owned blocks then equal G x.
    for pr in _problems():
        o = Oracle(pr)
        P = 3 if pr.n >= 6 else 2
        b = opart.slab_bounds(pr, P, o.cls)
        owners = opart.face_owner(pr, o.faces, b)
        x = np.random.default_rng(5).uniform(-1, 1, o.n_active)
        y_ref = o.apply(x)
        wins = [opart.window(pr, o.num, b, r) for r in range(P)]
        loc = []
        for r, win in enumerate(wins):
            xg = np.zeros(o.n_active)                        # only the window is known
            s = slice(win["offset"], win["offset"] + win["n_local"])
            xg[s] = x[s]
            loc.append(o.apply(xg, [ow == r for ow in owners])[s].copy())
        for r in range(P - 1):
            halo = loc[r][wins[r]["n_owned"]:]
            loc[r + 1][:wins[r + 1]["n_lower"]] += halo
        y = np.concatenate([loc[r][:wins[r]["n_owned"]] for r in range(P)])
        np.testing.assert_allclose(y, y_ref, rtol=0, atol=1e-13 * np.abs(y_ref).max())
        # the face subsets cover every face once
        assert sum(int(np.count_nonzero(ow == r)) for ow in owners for r in range(P)) == o.n_faces
