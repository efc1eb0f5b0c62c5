"""The paper's own evaluation of y = G x on the CPU (Kronecker form, numpy FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).  This module is not part of
the oracle's definition: the oracle never uses the tensor-product factorisation.
It is the paper-like CPU baseline that bench.py times beside the oracle, and
tests/test_baseline_kronecker.py checks it against the oracle's explicit face
matrices.

Sec. 2.4: on a face with normal a the face matrix factorises as
    G_F = sum_j c_j h^(2j-1) (M^h (x) ... (x) G^h_j (x) ...)  = h^(d-2) (M^ (x) ... (x) G^ (x) ...)
with the reference mass M^ on the tangential directions and the reference penalty
G^ = sum_j c_j g_j g_j^T along the normal (g_j: jump of the j-th derivative of the
2k+1 patch basis functions across the face of [0,1] u [1,2]), the rightmost factor
acting on the x index.  Sec. 2.5.1 applies it in three one-dimensional steps.  Here
each step is one large matrix product over all faces of an axis (BLAS threads).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from oracle.basis import gauss_legendre, gauss_lobatto_nodes, lagrange_derivative_at, lagrange_value


def reference_1d(k: int):
    """(M^, [g_1..g_k]) on the reference cell [0, 1] with Gauss-Lobatto nodes."""
    xi = gauss_lobatto_nodes(k)
    xq, wq = gauss_legendre(k + 1, 0.0, 1.0)
    val = np.array([[lagrange_value(xi, m, x) for x in xq] for m in range(k + 1)])
    mass = (val * wq) @ val.T
    g = np.zeros((k, 2 * k + 1))
    for j in range(1, k + 1):
        for b in range(2 * k + 1):
            v = 0.0
            if b <= k:
                v += lagrange_derivative_at(xi, b, 1.0, j)        # K- at its right end
            if b >= k:
                v -= lagrange_derivative_at(xi, b - k, 0.0, j)    # K+ at its left end
            g[j - 1, b] = v
    return mass, g


class KroneckerCPU:
    """y = G x by the factorised face operator, for a workloads.Problem and its Oracle
    (the oracle supplies the face list and the patch numbering)."""

    def __init__(self, pr, oracle):
        d, k = pr.dim, pr.degree
        self.pr, self.o = pr, oracle
        mass, g = reference_1d(k)
        c = np.asarray(pr.cweights(), dtype=np.float64)
        self.M = mass
        self.G = (g.T * c) @ g                                    # sum_j c_j g_j g_j^T
        self.scale = pr.h ** (d - 2)
        self.idx = [oracle.patch_index(a) for a in range(d)]

    def _along(self, U, axis, A):
        """Apply the 1D matrix A along `axis` (1 = x, ..., in an array [face, z, y, x])."""
        Ut = np.moveaxis(U, axis, -1)
        return np.moveaxis(Ut @ A.T, -1, axis)

    def apply(self, x: np.ndarray) -> np.ndarray:
        """The three one-dimensional steps as numpy matrix products (one per direction)."""
        pr, o = self.pr, self.o
        d, k = pr.dim, pr.degree
        x = np.asarray(x, dtype=np.float64)
        y = np.zeros(o.n_active)
        for a in range(d):
            idx = self.idx[a]
            if idx.shape[0] == 0:
                continue
            ext = [2 * k + 1 if b == a else k + 1 for b in range(d)]   # patch box, x first
            U = x[idx].reshape((idx.shape[0],) + tuple(reversed(ext)))  # [face, (z,) y, x]
            for b in range(d):
                ax = d - b                                         # array axis of direction b
                U = self._along(U, ax, self.G if b == a else self.M)
            y += np.bincount(idx.ravel(), weights=(self.scale * U).reshape(idx.shape).ravel(),
                             minlength=o.n_active)
        return y


class KroneckerOpenMP(KroneckerCPU):
    """The same factorised apply in C with OpenMP over faces (baselines/kron_cpu.c, built by
    baselines/build_c.py): the paper-like CPU baseline that bench.py times."""

    def __init__(self, pr, oracle, nthreads: int | None = None):
        super().__init__(pr, oracle)
        from . import build_c
        self.lib = C.CDLL(build_c.build())
        f = self.lib.kron_apply
        f.restype = C.c_int
        f.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.POINTER(C.c_int64)),
                      C.POINTER(C.POINTER(C.c_int64)), C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_double,
                      C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int64, C.c_int]
        try:
            cores = len(os.sched_getaffinity(0))
        except AttributeError:
            cores = os.cpu_count() or 1
        self.nthreads = nthreads or cores
        d = pr.dim
        # colour classes (i_a mod 3, i_t mod 2): faces of one class share no node
        self._idx, self._coff = [], []
        for a in range(d):
            lower = oracle.faces[a]
            tang = [b for b in range(d) if b != a]
            col = lower[:, a] % 3
            for i, b in enumerate(tang):
                col = col + (3 << i) * (lower[:, b] % 2)
            order = np.argsort(col, kind="stable")
            self._idx.append(np.ascontiguousarray(self.idx[a][order], dtype=np.int64))
            self._coff.append(np.searchsorted(col[order], np.arange(13)).astype(np.int64))
        self._nf = (C.c_int64 * 3)(*[self._idx[a].shape[0] for a in range(d)] + [0] * (3 - d))
        self._ptrs = (C.POINTER(C.c_int64) * 3)(*[a.ctypes.data_as(C.POINTER(C.c_int64)) for a in self._idx])
        self._cptrs = (C.POINTER(C.c_int64) * 3)(*[c.ctypes.data_as(C.POINTER(C.c_int64)) for c in self._coff])
        self._M = np.ascontiguousarray(self.M)
        self._G = np.ascontiguousarray(self.G)

    def apply(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(self.o.n_active)
        dp = C.POINTER(C.c_double)
        rc = self.lib.kron_apply(self.pr.dim, self.pr.degree, self._nf, self._ptrs, self._cptrs, self._M.ctypes.data_as(dp),
                                 self._G.ctypes.data_as(dp), float(self.scale), x.ctypes.data_as(dp),
                                 y.ctypes.data_as(dp), int(self.o.n_active), int(self.nthreads))
        if rc != 0:
            raise RuntimeError("kron_apply failed")
        return y
