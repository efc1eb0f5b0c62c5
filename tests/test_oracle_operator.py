"""Pins of the oracle's global operator, classifier and numbering.

* kink functions u = ((x_a - x_P)_+)^m q(tangential) lie in V_h; their only
  non-zero jump is the m-th normal derivative on the plane x_a = x_P, so
  x^T G x = c_m h^(2m-1) (m!)^2 * integral over the penalised faces of q^2
  (closed form from the definition of g_F, Sec. 2.2);
* G annihilates interpolants of global polynomials of degree <= k in each
  variable, and does not annihilate degree k+1;
* G is symmetric positive semidefinite;
* DoF counts of fully active meshes match the numbers the paper prints;
* cell classes agree with dense sampling of the level set.
"""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import Polynomial

from oracle import mesh as omesh
from oracle.ghost_penalty import Oracle
from paper_2503_00246_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _power_norm(o, iters=30, seed=0):
    v = np.random.default_rng(seed).standard_normal(o.n_active)
    lam = 0.0
    for _ in range(iters):
        w = o.apply(v)
        lam = np.linalg.norm(w)
        v = w / lam
    return lam


@pytest.mark.parametrize("dim,k,m,axis", [(2, 1, 1, 0), (2, 2, 1, 1), (2, 2, 2, 0), (2, 4, 3, 1),
                                          (3, 1, 1, 2), (3, 2, 2, 0), (3, 3, 1, 1), (3, 3, 3, 2)])
@pytest.mark.parametrize("paper_w", [False, True])
def test_kink_energy_closed_form(dim, k, m, axis, paper_w):
    n, h = 4, 0.37
    c = W.paper_weights(0.5, k) if paper_w else None
    pr = W.box_problem(dim, n, k, all_faces=True, lo=0.0, hi=n * h, weights=c)
    o = Oracle(pr)
    xyz = o.num.coords()
    xP = 2 * h                                  # an interior mesh plane along `axis`
    rng = np.random.default_rng(3 + m + 7 * k)
    tang = [a for a in range(dim) if a != axis]
    qs = [Polynomial(rng.uniform(-1, 1, k + 1)) for _ in tang]    # degree k per tangential axis
    u = np.maximum(xyz[:, axis] - xP, 0.0) ** m
    for t, q in zip(tang, qs):
        u = u * q(xyz[:, t])
    e = o.energy(u)
    # faces in the plane: every face of the all-faces box with normal `axis` at x_P
    integral = 1.0
    for q in qs:
        Q = (q * q).integ()
        integral *= Q(n * h) - Q(0.0)
    cm = pr.cweights()[m - 1]
    ref = cm * h ** (2 * m - 1) * math.factorial(m) ** 2 * integral
    # rounding scale: sum_F |x_F|^T |A_F| |x_F| (cancellation in high-order jumps)
    eabs = sum(float(np.einsum("fi,ij,fj->", np.abs(u[o.patch_index(a)]), np.abs(o.A(a)),
                               np.abs(u[o.patch_index(a)]))) for a in range(dim))
    tol = 1e-14 * eabs + 1e-13 * abs(ref)
    assert abs(e - ref) <= tol, (e, ref, eabs)
    assert tol < 1e-6 * abs(ref)      # the check stays sharp enough to see a dropped term
    # and the operator applied to u is orthogonal to every smooth (global polynomial) vector
    y = o.apply(u)
    assert abs(np.dot(y, np.ones_like(y))) <= 1e-11 * np.abs(y).sum()


@pytest.mark.parametrize("dim,k,n", [(2, 1, 16), (2, 2, 16), (2, 5, 12), (3, 1, 10), (3, 2, 10),
                                     (3, 3, 8), (3, 4, 6)])
def test_polynomial_annihilation(dim, k, n):
    pr = W.small_ball(dim, n, k, radius=0.66, seed=20 + k)
    o = Oracle(pr)
    assert o.n_faces > 0
    xyz = o.num.coords()
    rng = np.random.default_rng(k)
    # tensor degree <= k (Q_k contains P_k): reproduced exactly by FE_Q
    u = np.ones(o.n_active)
    for a in range(dim):
        u = u * Polynomial(rng.uniform(-1, 1, k + 1))(xyz[:, a])
    Gn = _power_norm(o)
    r = np.linalg.norm(o.apply(u))
    assert r <= 1e-12 * Gn * np.linalg.norm(u), (r, Gn)
    # degree k+1 along x is not in V_h: its interpolant has derivative jumps
    v = xyz[:, 0] ** (k + 1)
    assert np.linalg.norm(o.apply(v)) > 1e-9 * Gn * np.linalg.norm(v)


@pytest.mark.parametrize("dim,k", [(2, 3), (3, 2)])
def test_operator_symmetric_psd(dim, k):
    pr = W.small_ball(dim, 10, k, seed=40 + k)
    o = Oracle(pr)
    rng = np.random.default_rng(1)
    Gn = _power_norm(o)
    for _ in range(4):
        x = rng.uniform(-1, 1, o.n_active)
        z = rng.uniform(-1, 1, o.n_active)
        a, b = z @ o.apply(x), x @ o.apply(z)
        assert abs(a - b) <= 1e-13 * Gn * np.linalg.norm(x) * np.linalg.norm(z)
        assert x @ o.apply(x) >= -1e-13 * Gn * (x @ x)
        assert abs(x @ o.apply(x) - o.energy(x)) <= 1e-12 * Gn * (x @ x)


def test_full_mesh_dof_counts_match_paper():
    rows = np.loadtxt(os.path.join(GOLDEN, "paper_full_mesh_dofs.txt"), dtype=np.int64)
    for k, n, ndofs in rows:
        pr = W.box_problem(3, int(n), int(k), all_faces=False)
        cls = omesh.classify_cells(pr)
        num = omesh.Numbering(pr, cls)
        assert num.n_active == ndofs


def test_numbering_lexicographic_x_fastest():
    pr = W.small_ball(2, 8, 2, seed=3)
    o = Oracle(pr)
    xyz = o.num.coords()
    # sorted by (y, x): x fastest
    key = np.lexsort((xyz[:, 0], xyz[:, 1]))
    assert np.array_equal(key, np.arange(o.n_active))
    assert len(np.unique(xyz, axis=0)) == o.n_active
    # every active DoF lies in the closure of an active cell
    h = pr.h
    act = np.argwhere(o.cls != omesh.OUTSIDE)
    lo = pr.lo + act * h
    inside = np.zeros(o.n_active, dtype=bool)
    for c in lo:
        inside |= np.all((xyz >= c - 1e-12) & (xyz <= c + h + 1e-12), axis=1)
    assert inside.all()


@pytest.mark.parametrize("dim", [2, 3])
def test_ball_classification_against_sampling(dim):
    pr = W.small_ball(dim, 12 if dim == 3 else 24, 1, radius=0.61, seed=9)
    cls = omesh.classify_cells(pr)
    h = pr.h
    c = pr.centers[0, :dim]
    r = pr.radii[0]
    g = np.linspace(0.0, 1.0, 7)
    loc = np.stack(np.meshgrid(*([g] * dim), indexing="ij"), axis=-1).reshape(-1, dim)
    for idx in np.ndindex(*cls.shape):
        lo = pr.lo + np.array(idx) * h
        pts = lo + loc * h
        phi = r - np.linalg.norm(pts - c, axis=1)
        near = np.clip(c, lo, lo + h)                  # nearest point of the cell box
        far = np.where(np.abs(lo - c) > np.abs(lo + h - c), lo, lo + h)
        phimax = r - np.linalg.norm(near - c)
        phimin = r - np.linalg.norm(far - c)
        if cls[idx] == omesh.INSIDE:
            assert phi.min() > 0 and phimin > 0
        elif cls[idx] == omesh.OUTSIDE:
            assert phi.max() <= 0 and phimax <= 0
        else:
            assert phimin <= 0 < phimax


def test_gyroid_classification_against_sampling():
    pr = W.gyroid_3d(k=1, n=12)
    cls = omesh.classify_cells(pr)
    assert (cls == omesh.CUT).sum() > 0 and (cls == omesh.INSIDE).sum() > 0
    h = pr.h
    rng = np.random.default_rng(2)
    for idx in np.ndindex(*cls.shape):
        lo = pr.lo + np.array(idx) * h
        pts = lo + rng.uniform(0, 1, (64, 3)) * h
        phi = W.levelset_value(pr, pts)
        if cls[idx] == omesh.INSIDE:
            assert phi.min() > 0
        elif cls[idx] == omesh.OUTSIDE:
            assert phi.max() < 0


def test_ghost_faces_definition_brute_force():
    pr = W.small_ball(3, 9, 2, seed=5)
    o = Oracle(pr)
    cls = o.cls
    n = pr.n
    found = set()
    for a in range(3):
        for f in o.faces[a]:
            found.add((a, tuple(f)))
    ref = set()
    for idx in np.ndindex(n, n, n):
        for a in range(3):
            nb = list(idx)
            nb[a] += 1
            if nb[a] >= n:
                continue
            c0, c1 = cls[idx], cls[tuple(nb)]
            if c0 != omesh.OUTSIDE and c1 != omesh.OUTSIDE and (c0 == omesh.CUT or c1 == omesh.CUT):
                ref.add((a, idx))
    assert found == ref
