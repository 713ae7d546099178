"""Comparison helpers for the system product of Eq. AEFIEoutJ (test-side only).

The two block rows of the product differ in size by orders of magnitude on the test fixtures
(row 2 carries F D j, large where the equivalent current has a surface divergence; row 1 carries
j k0 L^A j + I_x e - (F D)^T L^Phi q), so one norm over [y1; y2] cannot see an error confined to
row 1. Each block row is compared against its own norm, and element by element against its own
largest entry."""
import numpy as np


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def max_rel(a, b):
    """max_i |a_i - b_i| / max_i |b_i|."""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def check_system(got, ref, ne, tol, elem_tol=None, rows=None):
    """Assert that both block rows of `got` match `ref` within tol (relative 2-norm of the block)
    and elem_tol (largest element error over the block's largest entry; 3 tol by default).
    `rows`: optional (edge rows, triangle rows) when only sampled rows of each block are given,
    in which case got/ref hold the sampled rows of row 1 followed by those of row 2."""
    elem_tol = 3.0 * tol if elem_tol is None else elem_tol
    got, ref = np.asarray(got), np.asarray(ref)
    split = ne if rows is None else len(rows[0])
    out = {}
    for name, sl in (("y1", slice(0, split)), ("y2", slice(split, None))):
        g, r = got[sl], ref[sl]
        e2, em = rel(g, r), max_rel(g, r)
        out[name] = (e2, em)
        assert e2 < tol, f"{name}: relative error {e2:.3e} above {tol:.1e}"
        assert em < elem_tol, f"{name}: largest element error {em:.3e} above {elem_tol:.1e}"
    return out
