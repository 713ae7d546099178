"""Surface impedance boundary condition (SIBC), the comparison model of Sec. I: the internal
problem of each conductor is replaced by the local Leontovich relation n x E = Z_s n x (n x H)
with Z_s = sqrt(mu / eps_c), and H_eq = 0. Test infrastructure (oracle), FP64.

In the variables of Eq. (AEFIEoutJ) (lengths in um, e = E / eta0) the relation tested with the
RWG functions reads G e = -(Z_s / eta0) I_x h, G the Gram matrix of the RWG functions, so the
SIBC model takes Zhat_i = -(Z_s / eta0) G_ii^{-1} I_x,ii and Yhat_i = 0 (j = h) in place of the
internal blocks of Eqs. (MFIEinZin) and (EFIEeqYeq); the external operators are unchanged.
"""
from __future__ import annotations

import numpy as np

from .operators import eps_rc, gram_matrix, ix_matrix
from .rwg import RWG


def sibc_blocks(rw: RWG, freq, sigma, mur=1.0):
    """Per-object (Zhat_i, Yhat_i) of the SIBC model (dense, FP64)."""
    G = gram_matrix(rw)
    ix = ix_matrix(rw)
    Zs, Ys = [], []
    for i, (a, b) in enumerate(rw.obj_edge_ranges()):
        zs = np.sqrt(mur / eps_rc(sigma[i], freq))  # Z_s / eta0
        Zs.append(-zs * np.linalg.solve(G[a:b, a:b].toarray(), ix[a:b, a:b].toarray()))
        Ys.append(np.zeros((b - a, b - a)))
    return Zs, Ys
