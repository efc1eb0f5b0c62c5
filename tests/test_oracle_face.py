"""Pins of the oracle's explicit face matrix.

Each check is independent of the oracle's own construction (Taylor-form
Lagrange derivatives at Gauss points): exact rational matrices for k = 1,
a Kronecker product of 1D matrices that the test builds with numpy Legendre
fits, an energy computed by fitting polynomials along the normal, and
structural properties (symmetry, semidefiniteness, rank, translation
invariance).
"""
import os

import numpy as np
import pytest
from numpy.polynomial import Legendre

from oracle.basis import gauss_legendre, gauss_lobatto_nodes
from oracle.ghost_penalty import Oracle, face_matrix
from paper_2503_00246_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lag_poly(nodes, m, a, b):
    """Lagrange polynomial of nodes[m] as a Legendre series fitted on [a, b]."""
    e = np.zeros(len(nodes))
    e[m] = 1.0
    return Legendre.fit(nodes, e, len(nodes) - 1, domain=[a, b])


def _mass_1d(k):
    xi = gauss_lobatto_nodes(k)
    ps = [_lag_poly(xi, m, 0.0, 1.0) for m in range(k + 1)]
    M = np.zeros((k + 1, k + 1))
    for a in range(k + 1):
        for b in range(k + 1):
            q = (ps[a] * ps[b]).integ()
            M[a, b] = q(1.0) - q(0.0)
    return M


def _jumps_1d(k):
    """g_j[b], j = 1..k, on the reference patch [0,1] u [1,2]."""
    xi = gauss_lobatto_nodes(k)
    lo = [_lag_poly(xi, m, 0.0, 1.0) for m in range(k + 1)]
    hi = [_lag_poly(1.0 + xi, m, 1.0, 2.0) for m in range(k + 1)]
    g = np.zeros((k, 2 * k + 1))
    for j in range(1, k + 1):
        for b in range(2 * k + 1):
            v = 0.0
            if b <= k:
                v += lo[b].deriv(j)(1.0)
            if b >= k:
                v -= hi[b - k].deriv(j)(1.0)
            g[j - 1, b] = v
    return g


def test_k1_closed_form_2d_and_3d():
    # k = 1: g_1 = [-1, 2, -1], M = [[1/3, 1/6], [1/6, 1/3]]; G_F = c_1 h^(d-2) (M x ... x g g^T)
    gg = np.array([[1.0, -2.0, 1.0], [-2.0, 4.0, -2.0], [1.0, -2.0, 1.0]])
    M = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    for h in (1.0, 0.25, 3.0):
        A = face_matrix(2, 1, h, 0, [0.7])
        np.testing.assert_allclose(A, 0.7 * np.kron(M, gg), rtol=1e-13, atol=1e-15)
        A = face_matrix(2, 1, h, 1, [0.7])
        np.testing.assert_allclose(A, 0.7 * np.kron(gg, M), rtol=1e-13, atol=1e-15)
        A = face_matrix(3, 1, h, 0, [0.7])
        np.testing.assert_allclose(A, 0.7 * h * np.kron(M, np.kron(M, gg)), rtol=1e-13, atol=1e-15)
        A = face_matrix(3, 1, h, 1, [0.7])
        np.testing.assert_allclose(A, 0.7 * h * np.kron(M, np.kron(gg, M)), rtol=1e-13, atol=1e-15)
        A = face_matrix(3, 1, h, 2, [0.7])
        np.testing.assert_allclose(A, 0.7 * h * np.kron(gg, np.kron(M, M)), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6, 8])
@pytest.mark.parametrize("paper_w", [False, True])
def test_kronecker_identity(dim, k, paper_w):
    if dim == 3 and k > 6:
        pytest.skip("covered in 2D; 3D k=8 face matrix is large")
    h = 0.3
    c = np.array(W.paper_weights(0.5, k) if paper_w else [0.5] * k)
    M = _mass_1d(k)
    g = _jumps_1d(k)
    # the j = 0 jump of continuous FE_Q vanishes (reading: the sum starts at j = 1)
    xi = gauss_lobatto_nodes(k)
    v0 = np.zeros(2 * k + 1)
    v0[k] = _lag_poly(xi, k, 0, 1)(1.0) - _lag_poly(1 + xi, 0, 1, 2)(1.0)
    assert np.abs(v0).max() < 1e-12
    G = sum(c[j] * np.outer(g[j], g[j]) for j in range(k))
    for axis in range(dim):
        A = face_matrix(dim, k, h, axis, c)
        fac = [G if a == axis else M for a in range(dim)]
        K = fac[-1]
        for f in reversed(fac[:-1]):
            K = np.kron(K, f)  # rightmost factor acts on x (fastest index)
        K = K * h ** (dim - 2)
        err = np.abs(A - K).max() / np.abs(K).max()
        assert err < 1e-10, (axis, err)


@pytest.mark.parametrize("dim,k", [(2, 1), (2, 3), (2, 6), (3, 2), (3, 3), (3, 4)])
def test_face_matrix_spsd_rank_translation(dim, k):
    # equilibrate the orders (|g_j| grows fast with j) so the rank gap is clean
    g = _jumps_1d(k)
    c = 1.0 / (g ** 2).sum(axis=1)
    A = face_matrix(dim, k, 1.0, 0, c)
    np.testing.assert_allclose(A, A.T, atol=1e-12 * np.abs(A).max())
    ev = np.linalg.eigvalsh(A)
    assert ev.min() > -1e-12 * ev.max()
    # rank k (k+1)^(d-1): one jump per order j and tangential basis function
    assert int((ev > 1e-9 * ev.max()).sum()) == k * (k + 1) ** (dim - 1)
    # the local matrix is the same on every face of a Cartesian mesh (Sec. 2.2)
    B = face_matrix(dim, k, 1.0, 0, c, origin=np.array([3.0, -2.0, 5.0])[:dim])
    np.testing.assert_allclose(A, B, rtol=1e-9, atol=1e-9 * np.abs(A).max())


def _brute_energy(dim, k, h, axis, c, xF):
    """x^T G_F x by fitting polynomials through nodal values (no Taylor forms)."""
    xi = gauss_lobatto_nodes(k)
    ext = [2 * k + 1 if a == axis else k + 1 for a in range(dim)]
    X = xF.reshape(ext[::-1]).transpose()          # X[i_x, i_y(, i_z)]
    X = np.moveaxis(X, axis, 0)                     # normal index first
    tang = [a for a in range(dim) if a != axis]
    nq = k + 3
    tq = [gauss_legendre(nq, 0.0, h) for _ in tang]
    tb = [_lag_poly(h * xi, m, 0.0, h) for m in range(k + 1)]
    e = 0.0
    for qidx in np.ndindex(*([nq] * len(tang))):
        wq = np.prod([tq[t][1][qidx[t]] for t in range(len(tang))])
        tv = [np.array([tb[m](tq[t][0][qidx[t]]) for m in range(k + 1)]) for t in range(len(tang))]
        line = X
        for t in range(len(tang)):
            line = np.tensordot(line, tv[t], axes=([1], [0]))   # contract one tangential index
        # line: values at the 2k+1 normal nodes for this tangential point
        plo = Legendre.fit(-h + h * xi, line[:k + 1], k, domain=[-h, 0.0])
        phi = Legendre.fit(h * xi, line[k:], k, domain=[0.0, h])
        for j in range(1, k + 1):
            jump = plo.deriv(j)(0.0) - phi.deriv(j)(0.0)
            e += c[j - 1] * h ** (2 * j - 1) * wq * jump ** 2
    return e


@pytest.mark.parametrize("dim,k,axis", [(2, 1, 0), (2, 2, 1), (2, 4, 0), (3, 1, 2), (3, 2, 0),
                                        (3, 3, 1)])
def test_face_energy_brute_force(dim, k, axis):
    rng = np.random.default_rng(5 + 10 * dim + k)
    h = 0.7
    c = rng.uniform(0.2, 1.0, k)
    A = face_matrix(dim, k, h, axis, c)
    for _ in range(3):
        x = rng.uniform(-1, 1, A.shape[0])
        e_ref = _brute_energy(dim, k, h, axis, c, x)
        e = x @ A @ x
        assert abs(e - e_ref) <= 1e-9 * abs(e_ref), (e, e_ref)


def test_patch_numbering_matches_paper_figure():
    rows = np.loadtxt(os.path.join(GOLDEN, "paper_patch_numbering_2d_k2.txt"), dtype=np.int64)
    pr = W.box_problem(2, 2, 2, all_faces=True)
    o = Oracle(pr)
    # lattice of a full 2x2-cell mesh, k = 2: 5 x 5 nodes numbered X + 5 Y
    idx = o.patch_index(0)
    f0 = np.where((o.faces[0][:, 0] == 0) & (o.faces[0][:, 1] == 0))[0][0]
    for i, i1, i2 in rows:
        assert idx[f0, i] == i1 + 5 * i2
