"""Pins of the oracle's mass + stiffness operator (closed forms and invariants)."""
import numpy as np
import pytest
from numpy.polynomial import Polynomial

from oracle import mesh as omesh
from oracle.cell_operator import CellOperator, cell_matrices
from paper_2503_00246_gb300 import workloads as W


def test_k1_closed_form():
    # k = 1: M_1D = h [[1/3, 1/6], [1/6, 1/3]], S_1D = (1/h) [[1, -1], [-1, 1]]
    for h in (1.0, 0.3):
        M1 = h * np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
        S1 = np.array([[1.0, -1.0], [-1.0, 1.0]]) / h
        M, K = cell_matrices(2, 1, h)
        np.testing.assert_allclose(M, np.kron(M1, M1), rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(K, np.kron(M1, S1) + np.kron(S1, M1), rtol=1e-13, atol=1e-15)
        M, K = cell_matrices(3, 1, h)
        np.testing.assert_allclose(M, np.kron(M1, np.kron(M1, M1)), rtol=1e-13, atol=1e-15)
        Kref = (np.kron(M1, np.kron(M1, S1)) + np.kron(M1, np.kron(S1, M1)) + np.kron(S1, np.kron(M1, M1)))
        np.testing.assert_allclose(K, Kref, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("dim,k,n", [(2, 2, 10), (2, 5, 6), (3, 1, 8), (3, 3, 6), (3, 4, 5)])
def test_volume_constants_and_polynomial_energies(dim, k, n):
    pr = W.small_ball(dim, n, k, radius=0.63, seed=60 + k)
    cls = omesh.classify_cells(pr)
    num = omesh.Numbering(pr, cls)
    op = CellOperator(pr, num, cls)
    ncell = int((cls != omesh.OUTSIDE).sum())
    vol = ncell * pr.h ** dim
    one = np.ones(num.n_active)
    # mass of the constant: the active volume; stiffness annihilates constants
    assert abs(one @ op.apply(one, 1.0, 0.0) - vol) <= 1e-12 * vol
    assert np.abs(op.apply(one, 0.0, 1.0)).max() <= 1e-11 * np.abs(op.K).max()
    # u = a . x: |grad u|^2 = |a|^2 on every cell
    xyz = num.coords()
    a = np.array([0.3, -1.2, 0.7])[:dim]
    u = xyz @ a
    assert abs(u @ op.apply(u, 0.0, 1.0) - (a @ a) * vol) <= 1e-11 * (a @ a) * vol
    # u = q(x) of degree <= k in x: integral of u^2 and of u'^2 over the active cells
    q = Polynomial(np.random.default_rng(k).uniform(-1, 1, k + 1))
    u = q(xyz[:, 0])
    act = np.argwhere(cls != omesh.OUTSIDE)
    lo = pr.lo + act[:, 0] * pr.h
    Q2, D2 = (q * q).integ(), (q.deriv() ** 2).integ()
    mass_ref = np.sum(Q2(lo + pr.h) - Q2(lo)) * pr.h ** (dim - 1)
    stiff_ref = np.sum(D2(lo + pr.h) - D2(lo)) * pr.h ** (dim - 1)
    assert abs(u @ op.apply(u, 1.0, 0.0) - mass_ref) <= 1e-11 * abs(mass_ref)
    assert abs(u @ op.apply(u, 0.0, 1.0) - stiff_ref) <= 1e-10 * abs(stiff_ref)


def test_symmetric_positive():
    pr = W.small_ball(3, 7, 3, seed=70)
    cls = omesh.classify_cells(pr)
    num = omesh.Numbering(pr, cls)
    op = CellOperator(pr, num, cls)
    rng = np.random.default_rng(3)
    x, z = rng.standard_normal((2, num.n_active))
    assert abs(z @ op.apply(x) - x @ op.apply(z)) <= 1e-12 * np.abs(x) @ np.abs(op.apply(np.abs(z)))
    assert x @ op.apply(x) > 0
