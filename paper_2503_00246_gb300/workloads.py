"""Seeded synthetic workloads for the ghost-penalty operator.

This module only describes problems and draws random inputs: the mesh box,
the level-set geometry, the polynomial degree and penalty weights, and the
seeded vectors x (and the polynomial used for the annihilation check).  It
holds none of the operator's arithmetic, so both the CUDA path and the CPU
oracle may import it.

Geometry follows the numerical experiments of the paper (Sec. 3): a Cartesian
box mesh cut by a ball (the single-ball throughput study) or by a denser
surface (the "many intersected cells" study), here a gyroid.

Seeds: problem ``p`` of workload ``w`` uses base seed ``250300246 + 1000*w + p``.
Independent streams are spawned from it with a numpy ``SeedSequence``:
spawn key 0 draws the geometry, 1 the operand vectors x, 2 the polynomial
coefficients, 3 the right-hand side b.  Every generator is numpy PCG64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 250300246

LS_BALLS = 1
LS_GYROID = 2
LS_CONST = 4


@dataclass
class Problem:
    """One ghost-penalty problem: mesh, level set, element degree, weights."""
    name: str
    dim: int
    n: int                      # cells per direction (uniform, equal h per axis)
    lo: float
    hi: float
    degree: int
    gamma: float = 0.5
    weights: list | None = None  # per-order weights c_1..c_k; None -> all gamma
    ls_kind: int = LS_BALLS
    centers: np.ndarray = field(default_factory=lambda: np.zeros((1, 3)))
    radii: np.ndarray = field(default_factory=lambda: np.array([0.7]))
    iso: float = 0.0            # gyroid: phi = sin x cos y + sin y cos z + sin z cos x - iso
    ls_value: float = 1.0       # constant level set (every cell inside when > 0)
    all_faces: bool = False     # treat every interior face of the active mesh as a penalised face
    seed: int = BASE_SEED
    stabilization: int = 0      # 0: ghost penalty; 1: macro patch (gamma, no per-order weights)

    @property
    def h(self) -> float:
        return (self.hi - self.lo) / self.n

    def cweights(self) -> np.ndarray:
        """Per-order weights c_j, j = 1..k (default: gamma for every order)."""
        if self.weights is None:
            return np.full(self.degree, float(self.gamma))
        w = np.asarray(self.weights, dtype=np.float64)
        assert w.shape == (self.degree,)
        return w

    def stream(self, key: int) -> np.random.Generator:
        return np.random.Generator(np.random.PCG64(
            np.random.SeedSequence(self.seed, spawn_key=(key,))))


def paper_weights(gamma: float, k: int) -> list:
    """c_j = gamma / (j!)^2, the factorial weighting of the ghost-penalty sum (Sec. 2.2)."""
    return [gamma / math.factorial(j) ** 2 for j in range(1, k + 1)]


def _seed(workload: int, p: int = 0) -> int:
    return BASE_SEED + 1000 * workload + p


def _ball(name, dim, n, lo, hi, k, radius, seed, gamma=0.5, weights=None) -> Problem:
    pr = Problem(name=name, dim=dim, n=n, lo=lo, hi=hi, degree=k, gamma=gamma,
                 weights=weights, ls_kind=LS_BALLS, seed=seed)
    off = pr.stream(0).uniform(-0.05, 0.05, dim)
    c = np.zeros((1, 3))
    c[0, :dim] = off
    pr.centers = c
    pr.radii = np.array([float(radius)])
    return pr


def disc_2d(k: int = 2, n: int = 32) -> Problem:
    """2D, 32x32 cells on [-1,1]^2, disc of radius 0.7 with a seeded centre offset."""
    return _ball(f"disc2d_n{n}_k{k}", 2, n, -1.0, 1.0, k, 0.7, _seed(1))


def ball_3d(k: int = 3, n: int = 64) -> Problem:
    """3D, 64^3 cells on [-1,1]^3, ball of radius 0.7 with a seeded centre offset."""
    return _ball(f"ball3d_n{n}_k{k}", 3, n, -1.0, 1.0, k, 0.7, _seed(2))


def ball_3d_sweep(k: int, n: int = 96) -> Problem:
    """3D degree sweep, 96^3 cells on [-1,1]^3, ball of radius 0.7 (same geometry for every k)."""
    return _ball(f"ball3d_sweep_n{n}_k{k}", 3, n, -1.0, 1.0, k, 0.7, _seed(3))


def gyroid_3d(k: int = 4, n: int = 128) -> Problem:
    """3D, 128^3 cells on [-pi,pi]^3, gyroid level set with iso value 0.3."""
    return Problem(name=f"gyroid3d_n{n}_k{k}", dim=3, n=n, lo=-math.pi, hi=math.pi,
                   degree=k, ls_kind=LS_GYROID, iso=0.3, seed=_seed(4))


def batched_3d(nprob: int = 64) -> list:
    """Independent 3D ball problems: n ~ U{16..96}, k ~ U{2..6}, r ~ U[0.4, 0.8]."""
    out = []
    for p in range(nprob):
        s = _seed(5, p)
        g = np.random.Generator(np.random.PCG64(np.random.SeedSequence(s, spawn_key=(0,))))
        n = int(g.integers(16, 97))
        k = int(g.integers(2, 7))
        r = float(g.uniform(0.4, 0.8))
        off = g.uniform(-0.05, 0.05, 3)
        pr = Problem(name=f"batch{p}_n{n}_k{k}", dim=3, n=n, lo=-1.0, hi=1.0, degree=k,
                     ls_kind=LS_BALLS, seed=s)
        pr.centers = off.reshape(1, 3).copy()
        pr.radii = np.array([r])
        out.append(pr)
    return out


def box_problem(dim: int, n: int, k: int, all_faces: bool = True, gamma: float = 0.5,
                weights=None, lo: float = 0.0, hi: float | None = None, seed: int = 7) -> Problem:
    """Every cell inside (constant positive level set); faces penalised when all_faces."""
    if hi is None:
        hi = float(n)
    return Problem(name=f"box{dim}d_n{n}_k{k}", dim=dim, n=n, lo=lo, hi=hi, degree=k,
                   gamma=gamma, weights=weights, ls_kind=LS_CONST, ls_value=1.0,
                   all_faces=all_faces, seed=seed)


def small_ball(dim: int, n: int, k: int, radius: float = 0.7, seed: int = 11,
               weights=None) -> Problem:
    return _ball(f"smallball{dim}d_n{n}_k{k}", dim, n, -1.0, 1.0, k, radius,
                 BASE_SEED + seed, weights=weights)


def levelset_value(pr: Problem, xyz: np.ndarray) -> np.ndarray:
    """phi at points (N x dim); positive inside.  Used for input checks only."""
    xyz = np.atleast_2d(xyz)
    if pr.ls_kind == LS_BALLS:
        vals = []
        for c, r in zip(pr.centers, pr.radii):
            vals.append(r - np.sqrt(((xyz - c[:pr.dim]) ** 2).sum(axis=1)))
        return np.max(np.stack(vals), axis=0)
    if pr.ls_kind == LS_GYROID:
        x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
        return (np.sin(x) * np.cos(y) + np.sin(y) * np.cos(z) + np.sin(z) * np.cos(x)) - pr.iso
    return np.full(xyz.shape[0], pr.ls_value)


def x_vectors(pr: Problem, n_active: int, nrhs: int = 1) -> np.ndarray:
    """Operand vectors x ~ U[-1,1], shape (nrhs, n_active), float64."""
    return pr.stream(1).uniform(-1.0, 1.0, (nrhs, n_active))


def rhs_vector(pr: Problem, n_active: int) -> np.ndarray:
    return pr.stream(3).uniform(-1.0, 1.0, n_active)


def poly_exponents(dim: int, deg: int) -> list:
    """Monomial exponents of total degree <= deg."""
    out = []
    if dim == 2:
        for a in range(deg + 1):
            for b in range(deg + 1 - a):
                out.append((a, b, 0))
    else:
        for a in range(deg + 1):
            for b in range(deg + 1 - a):
                for c in range(deg + 1 - a - b):
                    out.append((a, b, c))
    return out


def poly_coeffs(pr: Problem, deg: int | None = None) -> tuple:
    """Seeded coefficients of a random global polynomial of total degree <= deg."""
    deg = pr.degree if deg is None else deg
    ex = poly_exponents(pr.dim, deg)
    co = pr.stream(2).uniform(-1.0, 1.0, len(ex))
    return ex, co


def poly_eval(ex, co, xyz: np.ndarray) -> np.ndarray:
    """Evaluate sum_m co[m] * x^a y^b z^c at points (N x dim)."""
    xyz = np.atleast_2d(xyz)
    out = np.zeros(xyz.shape[0])
    for (a, b, c), cm in zip(ex, co):
        t = cm * xyz[:, 0] ** a * xyz[:, 1] ** b
        if c:
            t = t * xyz[:, 2] ** c
        out += t
    return out
