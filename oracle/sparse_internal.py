"""Sparse internal operators at high frequency (Sec. III-A, the third item of the internal
problem). Test infrastructure (oracle), FP64; only tests/ and the benchmark's CPU baseline use it.

When the skin depth delta = -1/Im k_i is small against an object, L_{k_i} and K_{k_i} couple a
basis function only to its near neighbours to any significant degree: the paper treats them as
sparse matrices, dropping physically distant interactions, and applies L^{-1} through a sparse
direct solver. The paper gives no cut-off. Reading adopted here:

* the pair (m, n) is kept iff the supports of f_m and f_n come within R_cut = CUT * delta of
  each other, CUT = 23 (the kernel factor e^{-R/delta} is below 1e-10 there);
* the support distance is bounded from below by
      d_mn = min over T in supp f_m, S in supp f_n of max(0, |c_T - c_S| - rho_T - rho_S),
  c the centroid and rho the largest centroid-to-vertex distance of a triangle, so every pair
  whose true distance is within R_cut is kept;
* e = Z_s h = -(1 / (j k0 eps_rc)) L_s^{-1} (K_s + I_x / 2) h, with L_s and K_s the kept entries
  (I_x couples only edges of a common triangle, at distance 0, and is kept whole), and
  L_s^{-1} applied by a sparse LU (SuperLU) as the library step.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .operators import dense_rwg, eps_rc, ix_matrix, k0_of, k_medium
from .rwg import RWG

CUT = 23.0


def tri_radius(rw: RWG) -> np.ndarray:
    """rho_T: largest distance from a triangle's centroid to its vertices."""
    X = rw.verts[rw.tris]
    return np.max(np.linalg.norm(X - rw.centroid[:, None, :], axis=2), axis=1)


def support_distance(rw: RWG, e0: int, e1: int) -> np.ndarray:
    """d_mn (lower bound of the distance between the supports of f_m and f_n), edges e0..e1."""
    c, rho = rw.centroid, tri_radius(rw)
    T = rw.et[e0:e1]
    n = e1 - e0
    D = np.full((n, n), np.inf)
    for a in range(2):
        for b in range(2):
            t, s = T[:, a], T[:, b]
            dc = np.linalg.norm(c[t][:, None, :] - c[s][None, :, :], axis=2)
            D = np.minimum(D, np.maximum(0.0, dc - rho[t][:, None] - rho[s][None, :]))
    return D


def skin_depth(k0, epsc, mur=1.0):
    return -1.0 / k_medium(k0, epsc, mur).imag


def pattern(rw: RWG, e0: int, e1: int, delta: float, cut: float = CUT) -> np.ndarray:
    """Kept pairs of the object's edges e0..e1 (boolean n x n)."""
    return support_distance(rw, e0, e1) <= cut * delta


class SparseZ:
    """e = Z_s h for one object: the sparse L_s, K_s + I_x/2 and the LU of L_s."""

    def __init__(self, rw: RWG, freq, sigma, e0: int, e1: int, ix=None, cut: float = CUT,
                 LK=None):
        k0 = k0_of(freq)
        self.epsc = eps_rc(sigma, freq)
        ki = k_medium(k0, self.epsc)
        self.delta = -1.0 / ki.imag
        self.mask = pattern(rw, e0, e1, self.delta, cut)
        ix = ix_matrix(rw) if ix is None else ix
        L, K = dense_rwg(rw, ki, ("L", "K"), e0, e1) if LK is None else LK
        self.L = sp.csc_matrix(np.where(self.mask, L, 0.0))
        self.B = sp.csr_matrix(np.where(self.mask, K, 0.0)) + 0.5 * ix[e0:e1, e0:e1]
        self.lu = spla.splu(self.L)
        self.alpha = -1.0 / (1j * k0 * self.epsc)

    @property
    def density(self) -> float:
        return float(self.mask.mean())

    def __call__(self, h):
        return self.alpha * self.lu.solve(self.B @ np.asarray(h, dtype=np.complex128))
