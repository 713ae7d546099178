"""Constraint preconditioner of the SLIM system. Test infrastructure (oracle), FP64.

The paper solves Eq. (AEFIEoutJ) by GMRES with the constraint preconditioner of the augmented
EFIE literature it cites (Sec. II-C), factorised by a sparse direct solver (Sec. IV-D); the
preconditioner's construction is not in the paper. Reading adopted here: the system of
Eq. (AEFIEoutJ) with its two dense external operators replaced by their near-field parts,
  P_c = [[j k0 L^A_near (I - C) + I_x Z,  -(F D)^T L^Phi_near],
         [(F D) (I - C),                  j k0 I             ]],
where L^A_near and L^Phi_near keep the exact Galerkin entries of the near pairs of the AIM (the
pairs whose anchors lie within r_near cells, across objects as well as within them) and drop
the rest, and Z and C = Y_eq Z stay exact (block diagonal over the objects). The second block
row, the discrete continuity equation that the augmented formulation adds as a constraint,
holds no external operator and is therefore kept exactly. P_c is sparse apart from the
objects' own dense blocks; it is factorised once by sparse LU (SuperLU, standing in for the
paper's MUMPS) and applied on the right, x = P_c^{-1} u.

When the near region covers every pair, P_c is the dense system itself.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .operators import fd_matrix, ix_matrix, k0_of
from .rwg import RWG


def block_diag_sparse(blocks, ranges, n):
    """The block-diagonal matrix of dense blocks placed on the diagonal ranges [a, b)."""
    rows, cols, vals = [], [], []
    for B, (a, b) in zip(blocks, ranges):
        r, c = np.meshgrid(np.arange(a, b), np.arange(a, b), indexing="ij")
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(np.asarray(B).ravel())
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def near_part(L_exact, pairs, n):
    """The exact entries of L on the near pairs (M, N), zero elsewhere."""
    M, N = pairs
    return sp.csr_matrix((L_exact[M, N], (M, N)), shape=(n, n))


def constraint_matrix(rw: RWG, freq, Zs, Ys, LA_near, LP_near):
    """P_c as a sparse matrix (blocks as in the module docstring)."""
    k0 = k0_of(freq)
    ne, nt = rw.ne, rw.nt
    ranges = rw.obj_edge_ranges()
    Z = block_diag_sparse(Zs, ranges, ne)
    C = block_diag_sparse([Y @ Zi for Y, Zi in zip(Ys, Zs)], ranges, ne)
    I = sp.identity(ne, dtype=np.complex128, format="csr")
    ix = ix_matrix(rw)
    fd = fd_matrix(rw)
    A11 = 1j * k0 * (LA_near @ (I - C)) + ix @ Z
    A12 = -(fd.T @ LP_near)
    A21 = fd @ (I - C)
    A22 = 1j * k0 * sp.identity(nt, dtype=np.complex128, format="csr")
    return sp.bmat([[A11, A12], [A21, A22]], format="csc")


class ConstraintPrecond:
    """x = P_c^{-1} u by one sparse LU factorisation."""

    def __init__(self, rw: RWG, freq, Zs, Ys, LA_near, LP_near):
        self.P = constraint_matrix(rw, freq, Zs, Ys, LA_near, LP_near)
        self.lu = spla.splu(self.P)

    @property
    def nnz(self):
        return int(self.P.nnz)

    def __call__(self, r):
        return self.lu.solve(np.asarray(r, dtype=np.complex128))
