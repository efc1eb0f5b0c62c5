"""Pins of the macro-patch oracle (oracle/macro_patch.py; Sec. 2.2 names the macro-patch
stabilisation beside the ghost penalty).

Reading: per face, gamma times the integral over each of the two cells of the square of
(the function there - the extension of the neighbour cell's polynomial into it).  The
checks: the k = 1 closed form (on the patch [0,1] u [1,2] the difference on K+ is
(t - 1)(v0 - 2 v1 + v2), so each side gives 1/3 of (v0 - 2 v1 + v2)^2), an independent
evaluation with monomial-basis polynomials and a different quadrature rule, annihilation of
global polynomials of tensor degree <= k, symmetry / positive semidefiniteness / rank, and the
null space shared with the ghost-penalty face matrix.
"""
import numpy as np
import pytest
from numpy.polynomial import polynomial as npoly

from oracle.basis import gauss_lobatto_nodes
from oracle.ghost_penalty import face_matrix
from oracle.macro_patch import face_matrix_macro


def _kron_x_fastest(fac):
    K = fac[-1]
    for f in reversed(fac[:-1]):
        K = np.kron(K, f)
    return K


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("h", [1.0, 0.25, 2.0])
def test_k1_closed_form(dim, h):
    gamma = 0.7
    M = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    g = np.array([1.0, -2.0, 1.0])
    G = (2.0 / 3.0) * np.outer(g, g)
    for axis in range(dim):
        A = face_matrix_macro(dim, 1, h, axis, gamma)
        K = gamma * h ** dim * _kron_x_fastest([G if a == axis else M for a in range(dim)])
        assert np.abs(A - K).max() <= 1e-13 * np.abs(K).max()


def _energy_monomial(dim, k, h, axis, x, gamma, nq):
    """gamma sum_K int_K (u_K - E u_K')^2 with each cell's polynomial found by solving a
    monomial Vandermonde system on its nodes, integrated with nq Gauss points per axis."""
    xi = gauss_lobatto_nodes(k)
    ext = [2 * k + 1 if a == axis else k + 1 for a in range(dim)]
    loc = np.array(list(np.ndindex(*ext[::-1])))[:, ::-1]
    def cell_poly(c):
        # coefficients of the tensor polynomial interpolating x on cell c (0: K-, 1: K+)
        nodes, vals = [], []
        for I, li in enumerate(loc):
            b = li[axis] - k * c
            if 0 <= b <= k:
                pt = [(-h + c * h + h * xi[b]) if a == axis else h * xi[li[a]] for a in range(dim)]
                nodes.append(pt)
                vals.append(x[I])
        nodes = np.array(nodes)
        V = npoly.polyvander2d(nodes[:, 0], nodes[:, 1], [k, k]) if dim == 2 else \
            npoly.polyvander3d(nodes[:, 0], nodes[:, 1], nodes[:, 2], [k, k, k])
        return np.linalg.solve(V, np.array(vals))
    coef = [cell_poly(0), cell_poly(1)]
    tq, wq = np.polynomial.legendre.leggauss(nq)
    e = 0.0
    for c in (0, 1):
        lo = [(-h + c * h) if a == axis else 0.0 for a in range(dim)]
        pts = [lo[a] + h * (tq + 1) / 2 for a in range(dim)]
        grids = np.meshgrid(*pts, indexing="ij")
        w = np.ones_like(grids[0])
        for a in range(dim):
            shp = [1] * dim
            shp[a] = nq
            w = w * (h * wq / 2).reshape(shp)
        P = [g.ravel() for g in grids]
        def ev(cf):
            if dim == 2:
                return npoly.polyvander2d(P[0], P[1], [k, k]) @ cf
            return npoly.polyvander3d(P[0], P[1], P[2], [k, k, k]) @ cf
        d = ev(coef[c]) - ev(coef[1 - c])
        e += gamma * float(np.sum(w.ravel() * d * d))
    return e


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 2), (2, 4), (3, 1), (3, 2)])
def test_energy_independent_evaluation(dim, k):
    rng = np.random.default_rng(17 + k)
    h, gamma = 0.4, 0.5
    for axis in range(dim):
        A = face_matrix_macro(dim, k, h, axis, gamma)
        x = rng.uniform(-1, 1, A.shape[0])
        ref = _energy_monomial(dim, k, h, axis, x, gamma, k + 3)
        assert abs(x @ A @ x - ref) <= 1e-10 * abs(ref)


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 3), (2, 5), (3, 1), (3, 2), (3, 3)])
def test_spsd_rank_annihilation_and_shared_null_space(dim, k):
    h = 0.3
    xi = gauss_lobatto_nodes(k)
    for axis in range(dim):
        A = face_matrix_macro(dim, k, h, axis, 0.5)
        P = A.shape[0]
        assert np.abs(A - A.T).max() <= 1e-13 * np.abs(A).max()
        ev = np.linalg.eigvalsh(A)
        assert ev.min() >= -1e-12 * ev.max()
        rank = int(np.sum(ev > 1e-9 * ev.max()))
        assert rank == k * (k + 1) ** (dim - 1)
        # global polynomials of tensor degree <= k are reproduced on both cells: no penalty
        ext = [2 * k + 1 if a == axis else k + 1 for a in range(dim)]
        loc = np.array(list(np.ndindex(*ext[::-1])))[:, ::-1]
        coords = np.stack([(-h + h * np.concatenate([xi, 1 + xi[1:]])[loc[:, a]]) if a == axis
                           else h * xi[loc[:, a]] for a in range(dim)], axis=1)
        rng = np.random.default_rng(3)
        for _ in range(3):
            cf = rng.normal(size=(k + 1,) * dim)
            xp = npoly.polyval2d(coords[:, 0], coords[:, 1], cf) if dim == 2 else \
                npoly.polyval3d(coords[:, 0], coords[:, 1], coords[:, 2], cf)
            assert np.linalg.norm(A @ xp) <= 1e-10 * ev.max() * np.linalg.norm(xp)
        # same null space as the ghost penalty: adding it does not raise the rank
        if P <= 400:
            Ag = face_matrix(dim, k, h, axis, np.full(k, 0.5))
            S = A / ev.max() + Ag / np.abs(Ag).max()
            es = np.linalg.eigvalsh(S)
            assert int(np.sum(es > 1e-9 * es.max())) == rank
