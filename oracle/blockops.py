"""Block-diagonal products (Sec. II-C: Z and Y_eq are block diagonal, one block per object).
Test infrastructure (oracle)."""
from __future__ import annotations

import numpy as np


def block_gemv(blocks, offsets, x):
    """y[o_i : o_i + n_i] = B_i x[o_i : o_i + n_i] for square blocks B_i (one or more RHS)."""
    y = np.zeros_like(np.asarray(x, dtype=np.complex128))
    for B, o in zip(blocks, offsets):
        n = B.shape[0]
        y[o:o + n] = B @ x[o:o + n]
    return y
