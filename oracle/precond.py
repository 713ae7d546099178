"""Block-diagonal preconditioner of the SLIM system. Test infrastructure (oracle), FP64.

The paper solves Eq. (AEFIEoutJ) with GMRES and the constraint preconditioner of Qian 2009
(Sec. II-C); that preconditioner's construction is not in the paper. Reading adopted here:
for each object i, the system of Eq. (AEFIEoutJ) restricted to that object's own unknowns
[h_i; q_i], with the exact (dense) external matrices of the object,
  A_ii = [[j k0 L^A_ii + (-j k0 L^A_ii Y_i + I_x,ii) Z_i,  -(F D)_ii^T L^Phi_ii],
          [(F D)_ii (I - Y_i Z_i),                        j k0 I              ]],
inverted densely; M_bd = blockdiag(A_ii^{-1}) is applied on the right (x = M_bd u). For one
object M_bd is the exact inverse of the dense system.
"""
from __future__ import annotations

import numpy as np

from .operators import dense_rwg, fd_matrix, ix_matrix, k0_of, pulse_entries
from .rwg import RWG


def object_blocks(rw: RWG, freq, Zs, Ys):
    """Dense A_ii for every object (returns list of (e0, e1, t0, t1, A_ii))."""
    k0 = k0_of(freq)
    ix = ix_matrix(rw)
    fd = fd_matrix(rw)
    out = []
    for i, ((e0, e1), (t0, t1)) in enumerate(zip(rw.obj_edge_ranges(), rw.obj_tri_ranges())):
        n, m = e1 - e0, t1 - t0
        LA = dense_rwg(rw, k0, "A", e0, e1)
        T, S = np.meshgrid(np.arange(t0, t1), np.arange(t0, t1), indexing="ij")
        LP = pulse_entries(rw, k0, T.ravel(), S.ravel()).reshape(m, m)
        Ix = ix[e0:e1, e0:e1].toarray()
        FD = fd[t0:t1, e0:e1].toarray()
        Z, Y = Zs[i], Ys[i]
        A11 = 1j * k0 * LA + (-1j * k0 * LA @ Y + Ix) @ Z
        A12 = -FD.T @ LP
        A21 = FD @ (np.eye(n) - Y @ Z)
        A22 = 1j * k0 * np.eye(m)
        out.append((e0, e1, t0, t1, np.block([[A11, A12], [A21, A22]])))
    return out


class BlockDiagPrecond:
    def __init__(self, rw: RWG, freq, Zs, Ys):
        self.ne = rw.ne
        self.blocks = [(e0, e1, t0, t1, np.linalg.inv(A)) for (e0, e1, t0, t1, A)
                       in object_blocks(rw, freq, Zs, Ys)]

    def __call__(self, r):
        r = np.asarray(r, dtype=np.complex128)
        u = np.zeros_like(r)
        ne = self.ne
        for e0, e1, t0, t1, Minv in self.blocks:
            v = np.concatenate([r[e0:e1], r[ne + t0:ne + t1]])
            w = Minv @ v
            u[e0:e1] = w[:e1 - e0]
            u[ne + t0:ne + t1] = w[e1 - e0:]
        return u
